"""The N > 1 path of bench.py on the CPU: replicas over gloo, world size 2.

Each rank times its own copy of the workload; the job's throughput is all
ranks' units over the slowest rank's time (max all-reduce), and the
reference arm runs on rank 0 only.  No GPU is used.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = 10.0 * (rank + 1)                  # rank 1 is the slow one
    slow = bench.slowest_rank_ms(local)
    out[rank] = (slow, bench.replica_value(1000, ws, slow))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    ws = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        slow, value = res[rank]
        assert slow == 20.0
        assert value == pytest.approx(2 * 1000 / 0.020)


def test_single_process_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(12.5) == 12.5
    assert bench.replica_value(500, 1, 12.5) == pytest.approx(500 / 0.0125)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(type("A", (), {"steps": 1, "warmup": 3})())
    assert capsys.readouterr().out == ""
