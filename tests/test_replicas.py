"""The multi-GPU mode of bench.py is replicas only (one independent copy of
the workload per rank, no collective on the data path): the job's time is
the slowest rank's and its throughput the units of all ranks over that time.
Checked with two gloo ranks on CPU."""
import importlib.util
import os
import socket

import pytest

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
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        # rank r took 10 + 5 r ms for 3e7 entries
        ms, value = bench.replica_value(10.0 + 5.0 * rank, 3.0e7, world, dist, device="cpu")
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_single_rank_is_plain_throughput():
    ms, value = _bench().replica_value(12.5, 1.0e9, 1)
    assert ms == 12.5 and value == pytest.approx(1.0e9 / 12.5e-3 / 1e9)


def test_two_gloo_ranks_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert sorted(out.keys()) == [0, 1]
    for r in (0, 1):
        ms, value = out[r]
        assert ms == 15.0
        assert value == pytest.approx(2 * 3.0e7 / 15.0e-3 / 1e9)
    del torch
