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


def test_oracle_sample_is_bounded_and_positive():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    w = synth.WORKLOADS["ic_rmat4k"]
    rate, S, cores, dt = bench.oracle_sample_rate(w.graph(), w, target_s=0.5)
    assert rate > 0 and S >= 16 and cores >= 1
    assert dt < 30.0  # the probe sizes the sample to about target_s


def test_count_roofline_from_stats():
    sys.path.insert(0, ROOT)
    import bench
    stats = [{"count_kernel_s": 0.01, "count_bytes": 30_000_000_000}, {"count_kernel_s": 0.01,
                                                                      "count_bytes": 30_000_000_000}]
    r = bench.count_roofline(stats, 6000.0)
    assert abs(r["achieved"] - 3000.0) < 1e-9 and abs(r["frac"] - 0.5) < 1e-12
    assert bench.count_roofline([{"count_kernel_s": 0.0, "count_bytes": 0}], 6000.0) is None
