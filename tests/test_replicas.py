"""The multi-process (replica) paths of bench.py on CPU: two gloo ranks agree on the
slowest rank's time, and the reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev = torch.device("cpu")
        bench.replica_barrier(world, dev)
        v = bench.replica_max(1.5 + rank, world, dev)
        bench.replica_barrier(world, dev)
        with open(os.path.join(out, f"r{rank}"), "w") as f:
            f.write(repr(v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    vals = [float(open(tmp_path / f"r{r}").read()) for r in range(world)]
    assert vals == [2.5, 2.5]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    torch = pytest.importorskip("torch")
    assert bench.replica_max(3.25, 1, torch.device("cpu")) == 3.25
    bench.replica_barrier(1, torch.device("cpu"))


def test_reference_arm_prints_only_on_rank_zero(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_oracle", lambda *a, **k: called.append(a))
    args = types.SimpleNamespace(workload="street_chain", warmup=3, steps=2, gpus=2)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.reference_main(args)
    assert buf.getvalue() == "" and not called
