#!/usr/bin/env python
"""Benchmark: end-to-end IMM over compressed RR sets on synthetic power-law graphs.

One step = one whole IMM run through the library (sampling fused with Huffman /
bitmap encoding for every estimation round and the final theta, greedy seed
selection on the compressed pool each round, FP64 bounds), with the graph
already resident in HBM.  The default workload is the twitter7-sized IC graph
(41,652,230 vertices, 1,468,365,182 edges, p ~ U[0, 0.1), k = 100, eps = 0.5).
Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hbx|reference]
                  [--workload ic_rmat42m] [--secondary wc_rmat1m] [--serving 200]

Besides the timed steps the line carries: the same IMM end to end from host
arrays (`e2e`), the plain one-launch-per-step form (`plain_form`), the
weighted-cascade 2^20-vertex workload measured the same way (`secondary`), the
serving stream (`serving`), the oracle on a bounded sample (`cpu_baseline`),
and rooflines of the dominant kernels.  Optional legs that would push the run
past --budget-s seconds are skipped and say so.

`--impl reference` times the CPU oracle (the plain statement of the method) on
the host, on a bounded sample of the same workload.  With N > 1 (torchrun)
every rank runs an independent replica (its own RR seed): the path has no data
exchange between independent IM queries, so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RR sets/s and end-to-end IMM s (bit-exact seeds); bytes/RR vertex; HBM GB/s % peak"
UNIT = "RR sets/s"
# workloads whose uncompressed (int32) pool would not fit one GPU: the plain
# form's comparison leg runs with the same Huffman + bitmap encoding there
INT32_TOO_BIG = {"ic_rmat42m"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


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


# ---------------------------------------------------------------------------
# oracle timing (the CPU baseline; test infrastructure, never on the product path)
# ---------------------------------------------------------------------------
def oracle_pool_rate(g, w, S, nthreads):
    """Oracle: sample sets [0, S) on nthreads host threads, then greedy k on
    them; returns (sets/s, seconds)."""
    import oracle
    model = oracle.IC if w.model == "IC" else oracle.LT
    pool = oracle.Pool(g, model, w.rr_seed)
    t0 = time.perf_counter()
    pool.extend(S, nthreads)
    pool.greedy(S, w.k)
    dt = time.perf_counter() - t0
    return S / dt, dt


def oracle_sample_size(g, w, target_s, cores):
    """Sets the oracle samples (with greedy) in about target_s on `cores`
    threads: doubling from 16 sets until a probe takes a second."""
    probe_n = 16
    while True:
        _, dt = oracle_pool_rate(g, w, probe_n, cores)
        if dt >= 1.0 or probe_n >= 2048:
            break
        probe_n *= 2
    return min(2_000_000, max(16, int(probe_n * target_s / max(dt, 1e-3))))


def oracle_baseline(g, w, target_s=15.0):
    cores = os.cpu_count() or 1
    if w.name == "ic_rmat42m":
        # a fifth of this graph's sets reach most of it (40-70 s each on one
        # core), the others are a single vertex: one set per core, all cores at
        # once (sets [0, cores) hold giant ones in about that share)
        S = cores
    else:
        S = oracle_sample_size(g, w, target_s, cores)
    rate, dt = oracle_pool_rate(g, w, S, cores)
    out = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": f"RR sets [0, {S}) of {w.name} sampled on {cores} threads, then greedy k={w.k} on them "
                     f"({dt:.1f} s)"}
    if w.name != "ic_rmat42m":
        S1 = max(16, S // (4 * cores))
        r1, d1 = oracle_pool_rate(g, w, S1, 1)
        out["single_thread"] = {"value": r1, "unit": UNIT, "sample": f"RR sets [0, {S1}) then greedy, one thread "
                                                                        f"({d1:.1f} s)"}
    return out


# ---------------------------------------------------------------------------
# rooflines
# ---------------------------------------------------------------------------
def sampler_roofline(stats, peak, peak_kind, wc):
    """Sampling fused with encoding, by the per-set algorithmic bytes: 8 per
    member (row_ptr pair), 4 per scanned edge for p (4 per member under the
    weighted cascade, whose p is a function of the target), 4 per live edge
    (col), plus the encoded bytes; over the sampling kernels' CUDA-event time."""
    ksec = sum(s["sample_kernel_s"] for s in stats)
    if ksec <= 0:
        return None
    per_p = (lambda s: 4 * s["rr_vertices"]) if wc else (lambda s: 4 * s["edges_scanned"])
    alg = sum(8 * s["rr_vertices"] + per_p(s) + 4 * s["edges_live"] + s["pool_bytes"] for s in stats)
    ach = alg / ksec / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
            "peak_kind": peak_kind, "kernel": "sampler: warp, shared-memory block and HBM block kernels, encode fused",
            "launches": int(sum(s["sample_kernel_launches"] for s in stats)), "kernel_s": ksec,
            "p_bytes": "4 per RR vertex (weighted cascade)" if wc else "4 per scanned edge"}


def search_roofline(stats, ceiling):
    """Bit-parallel search of the sets that outgrow shared memory: coin blocks
    drawn (one Philox4x32-10 per edge group and set that still needed coins)
    over the search's CUDA-event time, against the device's measured rate of
    the per-pair part of those blocks (hbx_philox_ceiling)."""
    ksec = sum(s["ms_kernel_s"] for s in stats)
    blocks = sum(s["ms_philox_blocks"] for s in stats)
    if ksec <= 0 or not ceiling:
        return None
    ach = blocks / ksec / 1e9
    return {"bound": "alu", "achieved": ach, "peak": ceiling / 1e9, "unit": "G coin blocks/s",
            "frac": ach / (ceiling / 1e9), "traffic": None, "peak_kind": "measured (hbx_philox_ceiling)",
            "kernel": "bit-parallel search (ms_light_kernel, ms_heavy_kernel, ms_compact_kernel per level)",
            "kernel_s": ksec, "blocks": blocks, "sets": int(sum(s["ms_sets"] for s in stats))}


def count_roofline(stats, peak):
    """Initial count passes (every counted set decoded or bit-plane summed once):
    bytes they read over their CUDA-event time."""
    cs = sum(s["count_kernel_s"] for s in stats)
    cb = sum(s["count_bytes"] for s in stats)
    if cs <= 0:
        return None
    ach = cb / cs / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "bytes_per_step": cb / len(stats), "kernel_s_per_step": cs / len(stats),
            "kernel": "count_items_kernel + bitmap_count_kernel (+ count_raw_kernel)"}


def dec_roofline(stats, peak):
    """Cover-and-decrement phases of the persistent selection: bytes of the
    covered sets the decrements read over the phases' time (globaltimer,
    barrier to barrier; the membership tests share that time)."""
    ds = sum(s["dec_s"] for s in stats)
    db = sum(s["dec_bytes"] for s in stats)
    if ds <= 0:
        return None
    ach = db / ds / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "bytes_per_step": db / len(stats), "s_per_step": ds / len(stats),
            "kernel": "select_persistent_kernel, cover-and-decrement phases"}


def selection_summary(stats):
    it = sum(s["select_iterations"] for s in stats)
    ks = sum(s["select_kernel_s"] for s in stats)
    if it == 0:
        return None
    return {"iterations_per_step": it / len(stats), "us_per_iteration": 1e6 * ks / it,
            "select_kernel_s_per_step": ks / len(stats)}


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


def timed_imms(hbx, tc, G, w, seed, opts, steps, flush):
    """`steps` IMMs, each bracketed by CUDA events on the library's stream, L2
    flushed (a 512 MB write) before each, outside the interval."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, stats, r = [], [], None
    for _ in range(steps):
        with torch.cuda.stream(tc.stream):
            flush.zero_()
        torch.cuda.synchronize()
        ev0.record(tc.stream)
        r = hbx.hbx_imm(tc.ctx, G, w.model, w.k, w.eps, w.ell, seed, opts)
        ev1.record(tc.stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        stats.append(r["stats"])
    return ms, stats, r


def pool_summary(s):
    return {"theta": s["theta"], "rr_vertices": s["rr_vertices"],
            "bytes_per_rr_vertex": s["pool_bytes"] / max(1, s["rr_vertices"]),
            "compression_vs_int32": s["raw_int32_bytes"] / max(1, s["pool_bytes"]),
            "uncoded_share": s["uncoded_vertices"] / max(1, s["rr_vertices"]),
            "sets": {"huffman": s["sets_huffman"], "bitmap": s["sets_bitmap"], "raw": s["sets_raw"],
                     "big": s["sets_big"], "bit_parallel": s["ms_sets"]},
            "skewness": s["skewness"], "density": s["density"]}


def plain_leg(hbx, tc, G, w, seed, steps, warmup, encode, flush, batched_ms, batched_r):
    """The plain one-launch-per-step form on the same workload and seed."""
    import numpy as np
    import torch
    torch.cuda.empty_cache()  # the plain form grows its heaps by copying (old + new at once)
    popts = hbx.hbx_default_options(encode=encode, form=0)
    for _ in range(warmup):
        hbx.hbx_imm(tc.ctx, G, w.model, w.k, w.eps, w.ell, seed, popts)
    pms, pstats, pr = timed_imms(hbx, tc, G, w, seed, popts, steps, flush)
    pmean = sum(pms) / len(pms)
    return {"ms_per_step": pmean, "value": pr["stats"]["theta"] / (pmean / 1000.0), "unit": UNIT,
            "steps": steps, "warmup": warmup, "encode": "huffman+bitmap" if encode else "int32",
            "batched_speedup": pmean / batched_ms, "seeds_equal": bool(np.array_equal(pr["seeds"], batched_r["seeds"])),
            "influence_equal": pr["influence"] == batched_r["influence"],
            "selection": selection_summary(pstats)}


def secondary_leg(hbx, synth, tc, name, steps, warmup, flush, peak, peak_kind, with_cpu):
    """A second workload measured the same way (timed IMMs, plain form,
    rooflines), for the weighted-cascade graph whose sets are small."""
    w = synth.WORKLOADS[name]
    g = w.graph()
    G = hbx.hbx_graph_create(tc.ctx, g)
    opts = hbx.hbx_default_options(encode=1, form=1)
    for _ in range(warmup):
        hbx.hbx_imm(tc.ctx, G, w.model, w.k, w.eps, w.ell, w.rr_seed, opts)
    ms, stats, r = timed_imms(hbx, tc, G, w, w.rr_seed, opts, steps, flush)
    mean = sum(ms) / len(ms)
    out = {"workload": name, "n": w.n, "m": w.m, "diffusion": w.model, "weights": w.weights, "k": w.k, "eps": w.eps,
           "steps": steps, "warmup": warmup, "ms_per_step": mean, "value": stats[-1]["theta"] / (mean / 1000.0),
           "unit": UNIT, **pool_summary(stats[-1]),
           "roofline": sampler_roofline(stats, peak, peak_kind, w.weights == "wc"),
           "count_roofline": count_roofline(stats, peak), "dec_roofline": dec_roofline(stats, peak),
           "selection": selection_summary(stats),
           "sample_kernel_s_per_step": sum(s["sample_kernel_s"] for s in stats) / len(stats)}
    out["plain_form"] = plain_leg(hbx, tc, G, w, w.rr_seed, max(3, steps // 3), 1, 0, flush, mean, r)
    if with_cpu:
        out["cpu_baseline"] = oracle_baseline(g, w)
    hbx.hbx_graph_destroy(G)
    return out


def serving_leg(hbx, synth, tc, count, rate=20.0, seed=3):
    """Poisson stream of IM queries over three resident graphs (the shapes of
    ic_rmat4k, wc_rmat1m and lt_rmat4m, each carrying IC probabilities and LT
    weights), model IC or LT, k in [10, 200], eps in {0.13, 0.2, 0.3, 0.5},
    served with continuous batching; RR pools stay resident across queries."""
    import numpy as np
    handles = []
    for name in ("ic_rmat4k", "wc_rmat1m", "lt_rmat4m"):
        w = synth.WORKLOADS[name]
        g = w.graph()
        if g.lt_weight is None:
            g.lt_weight = synth.lt_weights(g, w.graph_seed)
        if g.prob is None:
            g.prob = synth.ic_uniform(g, w.graph_seed, 0.1)
        handles.append(hbx.hbx_graph_create(tc.ctx, g))
        del g
    qs = synth.poisson_queries(seed=seed, count=count, rate_per_s=rate, graphs=[0, 1, 2])
    srv = hbx.hbx_server_create(tc.ctx, 4, 0)
    lat, fails, rejected = [], 0, []
    try:
        tickets = []
        t0 = time.perf_counter()
        for q in qs:
            while time.perf_counter() - t0 < q["t"]:
                time.sleep(0.0005)
            try:
                tickets.append((q, hbx.hbx_submit(tc.ctx, srv, handles[q["graph"]], q["model"], q["k"], q["eps"],
                                                  1.0, 7 + q["graph"])))
            except hbx.HbxError as e:
                # admission control: a query whose projected pool does not fit
                # the device is refused at submission
                rejected.append({"graph": q["graph"], "model": q["model"], "k": q["k"], "eps": q["eps"],
                                 "error": str(e)[:160]})
        for q, t in tickets:
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
    done = len(lat)
    lat = np.array(lat) if lat else np.zeros(1)
    qps = done / wall
    return {"queries": count, "completed": done, "failed": fails, "rejected": len(rejected),
            "rejected_queries": rejected[:8], "rate_per_s": rate, "queries_per_s": qps, "wall_s": wall,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_inflight": 4, "keeps_up": qps >= 0.95 * rate,
            "graphs": "ic_rmat4k, wc_rmat1m, lt_rmat4m shapes (IC probabilities and LT weights on each)"}


def run_reference(args, rank):
    import synth
    if rank != 0:
        return
    import oracle
    w = synth.WORKLOADS[args.workload]
    g = w.graph()
    model = oracle.IC if w.model == "IC" else oracle.LT
    times = []
    if w.name == "ic_rmat42m":
        # one RR set per step on one thread.  This graph's sets are either a
        # single vertex or reach 7.8 M vertices (about a fifth of them, 40-60 s
        # each on one core), and runs of consecutive ids can miss the giant ones,
        # so the ids are spread by a prime stride: 1000 + 7919 i for step i
        cores = 1
        ids = [1000 + 7919 * i for i in range(args.warmup + args.steps)]
        for i, j in enumerate(ids):
            t0 = time.perf_counter()
            oracle.rr_set(g, model, w.rr_seed, 0, j)
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
        S = 1
        sample = (f"one RR set of {w.name} per step, set ids 1000 + 7919 i (i = {args.warmup}..{args.warmup + args.steps - 1} "
                  f"timed), one thread")
    else:
        cores = os.cpu_count() or 1
        S = oracle_sample_size(g, w, min(15.0, 120.0 / max(1, args.steps + args.warmup)), cores)
        for i in range(args.warmup + args.steps):
            _, dt = oracle_pool_rate(g, w, S, cores)
            if i >= args.warmup:
                times.append(dt)
        sample = f"RR sets [0, {S}) of {w.name} sampled on {cores} threads then greedy k={w.k} on them, per step"
    tot_t = sum(times)
    value = S * len(times) / tot_t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "m": w.m, "diffusion": w.model, "weights": w.weights, "k": w.k,
                   "eps": w.eps, "ell": w.ell, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_hbx(args, rank, world, local_rank):
    import torch

    import paper_2208_00613_gb300 as hbx
    import synth

    t_start = time.perf_counter()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
    torch.cuda.set_device(local_rank)
    hbx.build()
    w = synth.WORKLOADS[args.workload]
    t0 = time.perf_counter()
    g = w.graph()
    synth_s = time.perf_counter() - t0
    seed = replica_seed(w.rr_seed, rank)
    tc = hbx.torch_context(local_rank)
    ctx = tc.ctx
    G = hbx.hbx_graph_create(ctx, g)
    opts = hbx.hbx_default_options(encode=args.encode, form=args.form)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{local_rank}")
    peak, peak_kind = peaks()
    ceiling = hbx.hbx_philox_ceiling(ctx)

    for _ in range(args.warmup):
        hbx.hbx_imm(ctx, G, w.model, w.k, w.eps, w.ell, seed, opts)
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    step_ms, stats, r = timed_imms(hbx, tc, G, w, seed, opts, args.steps, flush)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    sets = sum(s["theta"] for s in stats)
    if dist:
        total_ms_all, sets_all = reduce_over_ranks(total_ms, sets, f"cuda:{local_rank}")
    else:
        total_ms_all, sets_all = total_ms, float(sets)
    value = sets_all / (total_ms_all / 1000.0)
    imm_ms = total_ms / args.steps

    # end to end through the C ABI from host buffers: graph upload, IMM, results back
    e2e_ms, e2e_sets = [], 0
    h2d = graph_bytes(g)
    d2h = w.k * 4 + w.k * 8 + 8 + ctypes_sizeof_stats(hbx)
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = hbx.hbx_graph_create(ctx, g)
        r2 = hbx.hbx_imm(ctx, G2, w.model, w.k, w.eps, w.ell, seed, opts)
        hbx.hbx_graph_destroy(G2)
        e2e_ms.append(1000 * (time.perf_counter() - t0))
        e2e_sets += r2["stats"]["theta"]
    e2e_value = e2e_sets / (sum(e2e_ms) / 1000.0)

    if rank != 0:
        if dist:
            tdist.barrier()
        tc.close()
        return

    def left():
        return args.budget_s - (time.perf_counter() - t_start)

    def guarded(name, fn):
        try:
            return fn()
        except Exception as e:  # an optional leg never costs the bench line
            skipped[name] = f"error: {type(e).__name__}: {str(e)[:200]}"
            return None

    skipped = {}
    # the oracle baseline first (the contract's), then the optional legs in
    # order of importance, each only if its estimate fits the time budget
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        if left() > 150:
            cpu = guarded("cpu_baseline", lambda: oracle_baseline(g, w))
        else:
            skipped["cpu_baseline"] = "time budget"
    plain = None
    if not args.no_plain and args.form == 1:
        enc = args.plain_encode if args.plain_encode >= 0 else (1 if w.name in INT32_TOO_BIG else 0)
        pw = args.plain_warmup if args.plain_warmup >= 0 else (0 if w.name in INT32_TOO_BIG else 1)
        # the plain form ran 5.8x slower than the batched one at full size
        if left() > 6.2 * imm_ms / 1000.0 * (args.plain_steps + pw) + 30:
            plain = guarded("plain_form", lambda: plain_leg(hbx, tc, G, w, seed, args.plain_steps, pw, enc, flush,
                                                            imm_ms, r))
        else:
            skipped["plain_form"] = "time budget"
    serving = None
    if args.serving:
        if left() > 60:  # 200 queries at 20/s on three small graphs: about 30 s
            serving = guarded("serving", lambda: serving_leg(hbx, synth, tc, args.serving))
        else:
            skipped["serving"] = "time budget"
    secondary = None
    if args.secondary and world == 1:
        if left() > 40:  # 15 IMMs of ~25 ms plus its oracle sample: about 20 s
            secondary = guarded("secondary", lambda: secondary_leg(hbx, synth, tc, args.secondary, 12, 3, flush, peak,
                                                                   peak_kind, not args.no_cpu_baseline))
        else:
            skipped["secondary"] = "time budget"

    s0 = stats[-1]
    search = search_roofline(stats, ceiling)
    samp = sampler_roofline(stats, peak, peak_kind, w.weights == "wc")
    # the dominant kernel: the bit-parallel search when it holds most of the
    # sampling time, else the sampler as a whole
    dominant = search if search and search["kernel_s"] > 0.5 * samp["kernel_s"] else samp
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "m": w.m, "diffusion": w.model, "weights": w.weights, "k": w.k,
                   "eps": w.eps, "ell": w.ell, "encode": "huffman+bitmap" if args.encode else "int32",
                   "form": "persistent" if args.form else "plain", "parallelism": f"replicas{world}",
                   "l2": "flushed (512 MB write) between timed steps"},
        "imm_s": total_ms_all / args.steps / 1000.0,
        **pool_summary(s0),
        "traversed_edges_per_s": sum(s["edges_scanned"] for s in stats) / (total_ms / 1000.0),
        "warp_capacity": s0["warp_capacity"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": sum(e2e_ms) / len(e2e_ms), "steps": len(e2e_ms)},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "roofline": dominant,
        "sampler_roofline": samp,
        "search_roofline": search,
        "count_roofline": count_roofline(stats, peak),
        "dec_roofline": dec_roofline(stats, peak),
        "selection": selection_summary(stats),
        "phase_s_per_step": {"sample_kernels": sum(s["sample_kernel_s"] for s in stats) / len(stats),
                             "bit_parallel_search": sum(s["ms_kernel_s"] for s in stats) / len(stats),
                             "count": sum(s["count_kernel_s"] for s in stats) / len(stats),
                             "select_iterations": sum(s["select_kernel_s"] for s in stats) / len(stats)},
        "cpu_baseline": cpu,
        "plain_form": plain,
        "secondary": secondary,
        "serving": serving,
        "skipped": skipped or None,
        "synth_s": synth_s,
        "wall_s": time.perf_counter() - t_start,
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)
    if dist:
        tdist.barrier()
    tc.close()


def ctypes_sizeof_stats(hbx):
    import ctypes
    return ctypes.sizeof(hbx.hbx_stats)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hbx", choices=["hbx", "reference"])
    ap.add_argument("--workload", default="ic_rmat42m")
    ap.add_argument("--form", type=int, default=1)
    ap.add_argument("--encode", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison leg")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--plain-warmup", type=int, default=-1,
                    help="untimed plain-form IMMs before its timed ones (-1: 0 at full size, else 1)")
    ap.add_argument("--plain-encode", type=int, default=-1,
                    help="encoding of the plain-form leg (-1: Huffman + bitmap where an int32 pool would not fit "
                         "the GPU, else int32)")
    ap.add_argument("--secondary", default="wc_rmat1m", help="second workload measured in the same run ('' = none)")
    ap.add_argument("--serving", type=int, default=200, help="queries of the serving leg (0: skip)")
    ap.add_argument("--budget-s", type=float, default=1650.0,
                    help="optional legs that would run past this many seconds are skipped")
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
