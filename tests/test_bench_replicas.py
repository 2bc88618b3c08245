"""Host logic of bench.py's multi-GPU form (replicas only): the whole-job
value is all ranks' evaluations over the slowest rank's time, agreed by an
all-reduce MAX; under torchrun only rank 0 of the reference arm works.
World size 2 over gloo on the CPU."""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, seconds, steps, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        q.put((rank, bench.replica_throughput(seconds[rank], steps, world, dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_uses_the_slowest_rank():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    seconds, steps = [2.0, 2.5], 5
    procs = [ctx.Process(target=_worker, args=(r, 2, port, seconds, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [r for r, _ in got] == [0, 1]
    for _, v in got:
        assert v == pytest.approx(2 * steps / max(seconds))
    assert all(p.exitcode == 0 for p in procs)


def test_single_process_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(4.0, 8, 1) == pytest.approx(2.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = types.SimpleNamespace(warmup=3, steps=5, gpus=2, eig_fp32=False)
    assert bench.run_reference(args) == 0
