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
    g = w.graph()
    S = bench.oracle_sample_size(g, w, 0.5, 2)
    assert 16 <= S <= 2_000_000
    rate, dt = bench.oracle_pool_rate(g, w, S, 2)
    assert rate > 0 and dt < 30.0  # the probe sizes the sample to about target_s
    cb = bench.oracle_baseline(g, w, target_s=0.5)
    assert cb["value"] > 0 and cb["cores"] >= 1 and cb["kind"] == "oracle"
    assert cb["single_thread"]["value"] > 0 and cb["cpu_model"]


def test_rooflines_from_stats():
    sys.path.insert(0, ROOT)
    import bench
    s = {"sample_kernel_s": 0.5, "rr_vertices": 10, "edges_scanned": 100, "edges_live": 7, "pool_bytes": 50,
         "sample_kernel_launches": 3, "ms_kernel_s": 0.25, "ms_philox_blocks": 10**9, "ms_sets": 32,
         "dec_s": 0.001, "dec_bytes": 3_000_000, "select_iterations": 50, "select_kernel_s": 0.002}
    wc = bench.sampler_roofline([s], 6000.0, "measured", True)
    assert wc["achieved"] == (8 * 10 + 4 * 10 + 4 * 7 + 50) / 0.5 / 1e9
    ic = bench.sampler_roofline([s], 6000.0, "measured", False)
    assert ic["achieved"] == (8 * 10 + 4 * 100 + 4 * 7 + 50) / 0.5 / 1e9
    r = bench.search_roofline([s], 8e9)
    assert r["bound"] == "alu" and abs(r["achieved"] - 4.0) < 1e-12 and abs(r["frac"] - 0.5) < 1e-12
    d = bench.dec_roofline([s], 6000.0)
    assert abs(d["achieved"] - 3.0) < 1e-9
    assert abs(bench.selection_summary([s])["us_per_iteration"] - 40.0) < 1e-9


def test_count_roofline_from_stats():
    sys.path.insert(0, ROOT)
    import bench
    stats = [{"count_kernel_s": 0.01, "count_bytes": 30_000_000_000}, {"count_kernel_s": 0.01,
                                                                      "count_bytes": 30_000_000_000}]
    r = bench.count_roofline(stats, 6000.0)
    assert abs(r["achieved"] - 3000.0) < 1e-9 and abs(r["frac"] - 0.5) < 1e-12
    assert bench.count_roofline([{"count_kernel_s": 0.0, "count_bytes": 0}], 6000.0) is None


def test_serving_leg_counts_admission_refusals():
    """A query that admission control refuses at submission (its projected pool
    does not fit the device) is counted as refused; the leg still reports the
    other queries instead of ending the bench run."""
    import types
    sys.path.insert(0, ROOT)
    import bench

    class Err(RuntimeError):
        pass

    graphs = {}

    class FakeHbx:
        HbxError = Err

        @staticmethod
        def hbx_graph_create(ctx, g):
            graphs[len(graphs)] = g
            return len(graphs) - 1

        hbx_graph_destroy = staticmethod(lambda h: None)
        hbx_server_create = staticmethod(lambda ctx, inflight, budget: "srv")
        hbx_server_destroy = staticmethod(lambda srv: None)
        hbx_ticket_destroy = staticmethod(lambda t: None)

        @staticmethod
        def hbx_submit(ctx, srv, graph, model, k, eps, ell, seed):
            if eps == 0.13 and graph == 2:
                raise Err("ADMISSION: projected footprint exceeds the budget")
            return (graph, k)

        @staticmethod
        def hbx_wait(t, k):
            return 0, {"latency_s": 0.001 * (1 + t[1] % 7)}

    class G:
        lt_weight = None
        prob = None

    fake_synth = types.SimpleNamespace(
        WORKLOADS={n: types.SimpleNamespace(graph=lambda: G(), graph_seed=1)
                   for n in ("ic_rmat4k", "wc_rmat1m", "lt_rmat4m")},
        lt_weights=lambda g, s: "w", ic_uniform=lambda g, s, p: "p",
        poisson_queries=lambda seed, count, rate_per_s, graphs: [
            dict(t=0.0, graph=i % 3, model="IC", k=10 + i, eps=(0.13, 0.5)[i % 2]) for i in range(count)])
    out = bench.serving_leg(FakeHbx, fake_synth, types.SimpleNamespace(ctx=None), 12, rate=1e6)
    refused = sum(1 for i in range(12) if i % 3 == 2 and i % 2 == 0)
    assert out["rejected"] == refused and out["completed"] == 12 - refused and out["failed"] == 0
    assert all(r["eps"] == 0.13 and r["graph"] == 2 for r in out["rejected_queries"])
    assert out["p50_ms"] > 0 and out["queries_per_s"] > 0
