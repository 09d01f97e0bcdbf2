#!/usr/bin/env python
"""Benchmark: end-to-end IMM over compressed RR sets on synthetic power-law graphs.

One step = one whole IMM run through the library (sampling fused with Huffman /
bitmap encoding for every estimation round and the final theta, greedy seed
selection on the compressed pool each round, FP64 bounds), with the graph
already resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hbx|reference]
                  [--workload wc_rmat1m] [--form 1] [--encode 1]

`--impl reference` times the CPU oracle (the plain statement of the method) on
the host cores, on a bounded sample of the same workload.  With N > 1 (torchrun)
every rank runs an independent replica (its own RR seed): the path has no data
exchange between independent IM queries, so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RR sets/s and end-to-end IMM s (bit-exact seeds); bytes/RR vertex; HBM GB/s % peak"
UNIT = "RR sets/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def graph_bytes(g):
    b = g.row_ptr.nbytes + g.col.nbytes
    if g.prob is not None:
        b += g.prob.nbytes
    if g.lt_weight is not None:
        b += g.lt_weight.nbytes
    return b


def oracle_sample_rate(g, w, target_s=15.0, budget_sets=None):
    """Oracle throughput on a bounded sample: sample S sets of the workload on
    all host cores, then greedy k on them; returns (sets/s, S, cores, seconds).
    S is sized from a probe (doubling from 16 sets until a probe takes a
    second) so that the measured leg takes about target_s."""
    import oracle
    model = oracle.IC if w.model == "IC" else oracle.LT
    cores = os.cpu_count() or 1
    S = budget_sets
    if S is None:
        probe_n = 16
        while True:
            probe = oracle.Pool(g, model, w.rr_seed)
            t0 = time.perf_counter()
            probe.extend(probe_n, cores)
            probe.greedy(probe_n, w.k)
            dt = time.perf_counter() - t0
            del probe
            if dt >= 1.0 or probe_n >= 2048:
                break
            probe_n *= 2
        S = max(16, int(probe_n * target_s / max(dt, 1e-3)))
        S = min(S, 2_000_000)
    pool = oracle.Pool(g, model, w.rr_seed)
    t0 = time.perf_counter()
    pool.extend(S, cores)
    pool.greedy(S, w.k)
    dt = time.perf_counter() - t0
    return S / dt, S, cores, dt


def count_roofline(stats, peak):
    """Achieved bandwidth of the selections' count passes (decoding or
    bit-plane summing every counted set once): bytes they read over their
    CUDA-event time."""
    cs = sum(s["count_kernel_s"] for s in stats)
    cb = sum(s["count_bytes"] for s in stats)
    if cs <= 0:
        return None
    ach = cb / cs / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "bytes_per_step": cb / len(stats), "kernel_s_per_step": cs / len(stats),
            "kernel": "count_items_kernel + bitmap_count_kernel (+ count_raw_kernel)"}


def replica_seed(rr_seed, rank):
    """Philox key of rank `rank`'s replica: every rank solves its own instance."""
    return rr_seed + 1000 * rank


def reduce_over_ranks(total_ms, sets, device=None):
    """(slowest rank's timed interval, sets summed over ranks) over the default
    process group."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor([total_ms, float(sets)], dtype=torch.float64, device=device)
    mx = t.clone()
    tdist.all_reduce(mx, op=tdist.ReduceOp.MAX)
    sm = t.clone()
    tdist.all_reduce(sm, op=tdist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def serving_leg(hbx, synth, tc, resident, count, rate=20.0, seed=3):
    """Poisson stream of IM queries over three resident graphs (the shapes of
    ic_rmat4k, wc_rmat1m and lt_rmat4m, each carrying IC probabilities and LT
    weights), model IC or LT, k in [10, 200], eps in {0.13, 0.2, 0.3, 0.5},
    served with continuous batching; RR pools stay resident across queries."""
    import numpy as np
    handles = []
    for name in ("ic_rmat4k", "wc_rmat1m", "lt_rmat4m"):
        w = synth.WORKLOADS[name]
        g = resident.get(name) or w.graph()
        if g.lt_weight is None:
            g.lt_weight = synth.lt_weights(g, w.graph_seed)
        if g.prob is None:
            g.prob = synth.ic_uniform(g, w.graph_seed, 0.1)
        handles.append(hbx.hbx_graph_create(tc.ctx, g))
    qs = synth.poisson_queries(seed=seed, count=count, rate_per_s=rate, graphs=[0, 1, 2])
    srv = hbx.hbx_server_create(tc.ctx, 4, 0)
    lat, fails = [], 0
    try:
        tickets = []
        t0 = time.perf_counter()
        for q in qs:
            while time.perf_counter() - t0 < q["t"]:
                time.sleep(0.0005)
            tickets.append(hbx.hbx_submit(tc.ctx, srv, handles[q["graph"]], q["model"], q["k"], q["eps"], 1.0,
                                          7 + q["graph"]))
        for q, t in zip(qs, tickets):
            rc, res = hbx.hbx_wait(t, q["k"])
            hbx.hbx_ticket_destroy(t)
            if rc != 0:
                fails += 1
                continue
            lat.append(res["latency_s"])
        wall = time.perf_counter() - t0
    finally:
        hbx.hbx_server_destroy(srv)
        for h in handles:
            hbx.hbx_graph_destroy(h)
    lat = np.array(lat) if lat else np.zeros(1)
    return {"queries": count, "failed": fails, "rate_per_s": rate, "queries_per_s": (count - fails) / wall,
            "wall_s": wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_inflight": 4,
            "graphs": "ic_rmat4k, wc_rmat1m, lt_rmat4m shapes (IC probabilities and LT weights on each)"}


def run_reference(args, rank):
    import synth
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]
    g = w.graph()
    rates = []
    S = None
    cores = os.cpu_count() or 1
    for i in range(args.warmup + args.steps):
        rate, S, cores, dt = oracle_sample_rate(g, w, target_s=min(15.0, 120.0 / max(1, args.steps + args.warmup)),
                                                budget_sets=S)
        if i >= args.warmup:
            rates.append((rate, dt))
    tot_sets = S * len(rates)
    tot_t = sum(dt for _, dt in rates)
    value = tot_sets / tot_t
    sample = f"{S} RR sets of {w.name} sampled (all host cores) then greedy k={w.k} on them, per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / len(rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "m": w.m, "diffusion": w.model, "weights": w.weights, "k": w.k,
                   "eps": w.eps, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_hbx(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2208_00613_gb300 as hbx
    import synth

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    torch.cuda.set_device(local_rank)
    hbx.build()
    w = synth.WORKLOADS[args.workload]
    g = w.graph()
    seed = replica_seed(w.rr_seed, rank)
    tc = hbx.torch_context(local_rank)
    ctx = tc.ctx
    G = hbx.hbx_graph_create(ctx, g)
    opts = hbx.hbx_default_options(encode=args.encode, form=args.form)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{local_rank}")

    def one_step():
        return hbx.hbx_imm(ctx, G, w.model, w.k, w.eps, w.ell, seed, opts)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    step_ms, stats = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        with torch.cuda.stream(tc.stream):
            flush.zero_()  # L2 flush between timed steps, outside the timed interval
        torch.cuda.synchronize()
        ev0.record(tc.stream)
        r = one_step()
        ev1.record(tc.stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        stats.append(r["stats"])
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    sets = sum(s["theta"] for s in stats)
    if dist:
        total_ms_all, sets_all = reduce_over_ranks(total_ms, sets, f"cuda:{local_rank}")
    else:
        total_ms_all, sets_all = total_ms, float(sets)
    value = sets_all / (total_ms_all / 1000.0)

    # end to end through the C ABI from host buffers: graph upload, IMM, results back
    e2e_ms = []
    h2d = graph_bytes(g)
    d2h = w.k * 4 + w.k * 8 + 8 + ctypes_sizeof_stats(hbx)
    e2e_sets = 0
    for _ in range(max(1, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = hbx.hbx_graph_create(ctx, g)
        r = hbx.hbx_imm(ctx, G2, w.model, w.k, w.eps, w.ell, seed, opts)
        hbx.hbx_graph_destroy(G2)
        e2e_ms.append(1000 * (time.perf_counter() - t0))
        e2e_sets += r["stats"]["theta"]
    e2e_value = e2e_sets / (sum(e2e_ms) / 1000.0)

    if rank != 0:
        if dist:
            tdist.barrier()
        tc.close()
        return
    # the plain one-launch-per-step form (int32 sets, block per set, selection
    # launched round by round) on the same workload and seed, same timing rules
    plain = None
    if not args.no_plain and args.form == 1:
        # return the batched pools' memory, cached by torch's allocator, to the
        # device: the plain form grows its heaps by copying (old + new at once)
        torch.cuda.empty_cache()
        popts = hbx.hbx_default_options(encode=args.plain_encode, form=0)
        for _ in range(args.plain_warmup):
            hbx.hbx_imm(ctx, G, w.model, w.k, w.eps, w.ell, seed, popts)
        pms, pr = [], None
        for _ in range(args.steps):
            with torch.cuda.stream(tc.stream):
                flush.zero_()
            torch.cuda.synchronize()
            ev0.record(tc.stream)
            pr = hbx.hbx_imm(ctx, G, w.model, w.k, w.eps, w.ell, seed, popts)
            ev1.record(tc.stream)
            ev1.synchronize()
            pms.append(ev0.elapsed_time(ev1))
        pmean = sum(pms) / len(pms)
        plain = {"ms_per_step": pmean, "value": pr["stats"]["theta"] / (pmean / 1000.0), "unit": UNIT,
                 "encode": "huffman+bitmap" if args.plain_encode else "int32",
                 "batched_speedup": pmean / (total_ms / args.steps), "warmup": args.plain_warmup,
                 "seeds_equal": bool(np.array_equal(pr["seeds"], r["seeds"])),
                 "influence_equal": pr["influence"] == r["influence"]}
    serving = None
    if args.serving:
        serving = serving_leg(hbx, synth, tc, {w.name: g}, args.serving)
    # roofline of the dominant kernel (sampling fused with encoding)
    peak, peak_kind = peaks()
    alg_bytes = sum(8 * s["rr_vertices"] + 4 * s["edges_scanned"] + 4 * s["edges_live"] + s["pool_bytes"]
                    for s in stats)
    ksec = sum(s["sample_kernel_s"] for s in stats)
    klaunch = sum(s["sample_kernel_launches"] for s in stats)
    achieved = alg_bytes / ksec / 1e9 if ksec > 0 else 0.0
    traffic = None
    prof = os.path.join(ROOT, "profiles", "sample_kernel_traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                pj = json.load(f)
            if pj.get("workload") == w.name and pj.get("source_hash") == source_hash():
                traffic = pj.get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    s0 = stats[-1]
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, S, cores, dt = oracle_sample_rate(g, w)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{S} RR sets of {w.name} sampled then greedy k={w.k} on them ({dt:.1f} s)"}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "m": w.m, "diffusion": w.model, "weights": w.weights, "k": w.k,
                   "eps": w.eps, "ell": w.ell, "encode": "huffman+bitmap" if args.encode else "int32",
                   "form": "persistent+graph" if args.form else "plain", "parallelism": f"replicas{world}",
                   "l2": "flushed (512 MB write) between timed steps"},
        "imm_s": total_ms_all / args.steps / 1000.0,
        "theta": s0["theta"], "rr_vertices": s0["rr_vertices"],
        "bytes_per_rr_vertex": s0["pool_bytes"] / max(1, s0["rr_vertices"]),
        "compression_vs_int32": s0["raw_int32_bytes"] / max(1, s0["pool_bytes"]),
        "traversed_edges_per_s": sum(s["edges_scanned"] for s in stats) / (total_ms / 1000.0),
        "sets": {"huffman": s0["sets_huffman"], "bitmap": s0["sets_bitmap"], "raw": s0["sets_raw"],
                 "big": s0["sets_big"]},
        "skewness": s0["skewness"], "density": s0["density"], "warp_capacity": s0["warp_capacity"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": sum(e2e_ms) / len(e2e_ms)},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "sampler: warp, shared-memory block and HBM block kernels, encode fused",
                     "launches": klaunch, "kernel_s": ksec},
        "count_roofline": count_roofline(stats, peak),
        "cpu_baseline": cpu,
        "plain_form": plain,
        "serving": serving,
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)
    if dist:
        tdist.barrier()
    tc.close()


def ctypes_sizeof_stats(hbx):
    import ctypes
    return ctypes.sizeof(hbx.hbx_stats)


def source_hash():
    """Hash of the sampler kernels' sources (their device code and launchers):
    a stored DRAM-traffic capture is used only while these are unchanged."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2208_00613_gb300", "csrc")
    for f in ("common.cuh", "internal.h", "sample.cu", "msbfs.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hbx", choices=["hbx", "reference"])
    ap.add_argument("--workload", default="wc_rmat1m")
    ap.add_argument("--form", type=int, default=1)
    ap.add_argument("--encode", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison leg")
    ap.add_argument("--serving", type=int, default=0, help="queries of the serving leg (0: skip)")
    ap.add_argument("--plain-warmup", type=int, default=1, help="untimed plain-form IMMs before its timed ones")
    ap.add_argument("--plain-encode", type=int, default=0,
                    help="encoding of the plain-form leg (1 where an int32 pool would not fit the GPU)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    run_hbx(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
