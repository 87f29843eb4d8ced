"""The multi-GPU path of bench.py is replicas only (independent instances per
rank, no data-path collective): the job's step time is the slowest rank's, and
the throughput counts every rank's solves. Checked with two gloo ranks on CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench = _bench()
        ms_local = [2.0, 5.0][rank]  # rank 1 is the slower replica
        out[rank] = bench.replica_throughput(ms_local, world)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 5.0
        assert value == pytest.approx(world * 1000.0 / 5.0)


def test_single_process_is_its_own_replica():
    ms, value = _bench().replica_throughput(4.0, 1)
    assert ms == 4.0 and value == pytest.approx(250.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench = _bench()

    class Args:
        steps, warmup = 1, 0

    assert bench.run_reference(Args()) == 0  # returns before touching the oracle
