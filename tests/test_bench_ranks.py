"""Host logic of bench.py's multi-rank path, on CPU ranks over gloo: each rank
runs an independent replica (its own Philox key), the reported interval is the
slowest rank's and the reported sets are summed over ranks."""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    import bench
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = [120.0, 95.5][rank]
    sets = [45579, 45601][rank]
    q.put((rank, bench.reduce_over_ranks(ms, sets), bench.replica_seed(7, rank)))
    tdist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, (ms, sets), seed in out:
        assert ms == 120.0  # slowest rank
        assert sets == 45579 + 45601
    assert out[0][2] != out[1][2]  # independent replicas


def test_reference_arm_other_ranks_do_nothing(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload = "ic_rmat4k"
        steps = 1
        warmup = 0
        gpus = 2
    bench.run_reference(A(), rank=1)
    assert capsys.readouterr().out == ""
