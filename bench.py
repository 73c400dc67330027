#!/usr/bin/env python
"""Benchmark of RECEIPT tip decomposition on one GB300.

Workload: the Chung-Lu bipartite graph with |U| = 1,000,000, |V| = 200,000,
10,000,000 distinct edges, U-degree exponent 2.5 and V-degree exponent 2.1
(largest expected V degree 50,000), seed 2; the U side is decomposed.

One step = one whole pass of the hot path on the device: graph build
(deduplication, degree relabelling, two-sided CSR), per-vertex butterfly
counting (Algorithm 1), coarse-grained range peeling (Algorithm 3) and
fine-grained subset peeling (Algorithm 4), from an edge list already in HBM
to tip numbers in HBM.

Metric: wedges/s, where the wedge count of a step is the graph's bottom-up
peeling wedge count sum_{v in V} d_v (d_v - 1) (the work Algorithm 2 does; a
property of the graph, the same for every implementation), divided by the
step's device time. Seconds per step, the wedges the kernels actually walked
and the roofline fraction of the dominant kernel are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank decomposes its own copy of
the graph (the path has no exchange step: replicas only); the value is the
wedges of all ranks divided by the slowest rank's time.

--impl reference times the CPU oracle (sequential bottom-up peeling, test
infrastructure) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "wedges/s and end-to-end tip-decomp seconds on 1 GB300 (bit-exact); HBM roofline frac"
WORKLOAD = "chung-lu |U|=1M |V|=200k m=10M gamma 2.5/2.1 seed 2, U side"
CPU_SAMPLE_WEDGES = 1_500_000_000  # peel wedges per oracle sample (~10-20 s on one core)

# DRAM traffic of the dominant kernel from one full-size ncu capture, as DRAM
# bytes per algorithmic byte of the captured launch (scaled to the average
# launch of the timed step), keyed by kernel name; valid only while the peel
# kernels' sources (PEEL_SOURCES) hash to the recorded digest. k_cd_update_cta: CD round 4 of the
# 10M-edge Chung-Lu workload, 49.26 MB of DRAM for ~971 MB algorithmic.
NCU_TRAFFIC = {"k_cd_update_cta": {"src": "c1a903e285db3254", "dram_per_alg_byte": 0.0507}}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest of the ranks' values of x (x itself without a process
    group): the slowest replica's time decides the whole job's time."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job rate of `world` replicas that each process units_per_rank,
    timed by the slowest one."""
    return units_per_rank * world / seconds


def _rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# sources the coarse-grained peel kernels are compiled from
PEEL_SOURCES = ("cd.cu", "engine.cuh", "common.cuh", "internal.cuh")


def _src_digest(files=PEEL_SOURCES):
    """Digest of the named kernel sources (a recorded ncu traffic figure holds
    while the kernel's sources are unchanged)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2010_08695_gb300", "csrc")
    for f in sorted(files):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def load_workload():
    import synth
    eu, ev, nu, nv, side = synth.workload_graph(synth.CHUNG_LU_10M)
    dv = np.bincount(ev, minlength=nv).astype(np.int64)
    du = np.bincount(eu, minlength=nu).astype(np.int64)
    d_other = dv if side == 0 else du
    wedges = int((d_other * (d_other - 1)).sum())
    return eu, ev, nu, nv, side, wedges


def cpu_baseline(eu, ev, nu, nv, side, sample_wedges=CPU_SAMPLE_WEDGES, counts=None):
    """Oracle on a bounded sample: sequential bottom-up peeling of the same
    graph from its exact initial supports, stopped after `sample_wedges`."""
    import oracle
    t0 = time.perf_counter()
    if counts is None:
        counts = oracle.count_2hop(eu, ev, nu, nv)[side]
    t_count = time.perf_counter() - t0
    _, st = oracle.bup_from_counts(eu, ev, nu, nv, side, counts, max_wedges=sample_wedges)
    rate = st["wedges"] / st["seconds_peel"] if st["seconds_peel"] > 0 else 0.0
    return {"value": rate, "unit": "wedges/s", "cores": 1, "kind": "oracle",
            "sample": (f"sequential bottom-up peel (Algorithm 2, radix heap) of the benchmark "
                       f"graph from its exact initial supports, stopped after {st['wedges']} "
                       f"wedges / {st['peeled']} vertices in {st['seconds_peel']:.1f} s on one "
                       f"core; the initial support count took {t_count:.1f} s on "
                       f"{oracle.num_threads()} OpenMP threads and is not in the rate")}, counts


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    import oracle
    eu, ev, nu, nv, side, wedges = load_workload()
    counts = oracle.count_2hop(eu, ev, nu, nv)[side]
    sample = max(1, CPU_SAMPLE_WEDGES // 3)
    for _ in range(args.warmup):
        oracle.bup_from_counts(eu, ev, nu, nv, side, counts, max_wedges=sample // 10)
    rates, secs = [], []
    for _ in range(args.steps):
        _, st = oracle.bup_from_counts(eu, ev, nu, nv, side, counts, max_wedges=sample)
        rates.append(st["wedges"] / st["seconds_peel"])
        secs.append(st["seconds_peel"])
    value = statistics.mean(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "wedges/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nu": nu, "nv": nv, "m": int(len(eu)),
                       "side": "U", "wedges_bup": wedges,
                       "sample": f"{sample} peel wedges per step"},
            "cpu_baseline": {"value": value, "unit": "wedges/s", "cores": 1, "kind": "oracle",
                             "sample": f"sequential bottom-up peel of the benchmark graph from "
                                       f"its exact initial supports, {sample} wedges per step"},
            "e2e": {"value": value, "unit": "wedges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = _rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2010_08695_gb300 as R
    R.load()
    eu, ev, nu, nv, side, wedges = load_workload()
    n_side = nu if side == 0 else nv
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    eu_d = torch.from_numpy(eu).to(dev)
    ev_d = torch.from_numpy(ev).to(dev)
    tip = torch.empty(n_side, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    last_trace = []

    def step(timing):
        g = R.Graph(eu_d, ev_d, nu, nv, stream=stream)
        g.tip_decompose(side, P=args.P, timing=timing, out=tip, stream=stream,
                        round_graphs=args.round_graphs, huc=args.huc,
                        huc_factor_1024=args.huc_factor_1024)
        st = g.stats()
        if args.trace:
            last_trace[:] = g.trace()
        g.close()
        return st

    for _ in range(max(3, args.warmup)):
        step(True)
    barrier()
    times, stats = [], []
    launches0 = R.receipt_kernel_launches()
    with ClockSampler(local) as clk:
        barrier()
        for _ in range(args.steps):
            flush.fill_(1.0)  # evicts L2 between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats.append(step(True))
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        barrier()
    launches = R.receipt_kernel_launches() - launches0
    if args.trace and rank == 0:
        with open(args.trace, "w") as f:
            json.dump(last_trace, f)
    ms = max_over_ranks(statistics.mean(times), dist, dev)
    value = replica_rate(wedges, world, ms / 1e3)
    tips = R.as_u64(tip)

    # end to end through the C ABI with host buffers, with the options the
    # device-timed steps used (the shape class's tuned values)
    from paper_2010_08695_gb300 import autotune
    g0 = R.Graph(eu_d, ev_d, nu, nv, stream=stream)
    tuned = autotune.lookup(g0.shape_class(side)) or {}
    g0.close()
    e2e_opt = {"warp_max_w": tuned.get("warp_max_w", 0),
               "slice_min_w": tuned.get("slice_min_w", 0),
               "dgm_frac_1024": tuned.get("dgm_frac_1024", 0), "huc": args.huc,
               "huc_factor_1024": args.huc_factor_1024, "round_graphs": args.round_graphs}
    e2e_P = args.P or tuned.get("P", 150)
    eu_h = torch.from_numpy(eu).pin_memory().numpy()
    ev_h = torch.from_numpy(ev).pin_memory().numpy()
    tip_h = torch.empty(n_side, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
    R.receipt_tip_decompose_host(eu_h, ev_h, nu, nv, side, P=e2e_P, out=tip_h, **e2e_opt)
    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        barrier()
        t0 = time.perf_counter()
        R.receipt_tip_decompose_host(eu_h, ev_h, nu, nv, side, P=e2e_P, out=tip_h, **e2e_opt)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e_t), dist, dev)
    e2e_ok = bool(np.array_equal(tip_h, tips))

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # roofline of the dominant peel kernel (tier with the most device time)
    st = stats[-1]
    names = ["k_cd_update_warp", "k_cd_update_cta", "k_cd_update_global", "k_cd_update_slice",
             "k_cd_update_dense"]
    tier = max(range(5), key=lambda t: st["ms_peel"][t])
    lau = max(1, st["peel_launches"][tier])
    alg_bytes = (4 * st["peel_wedges"][tier] + 16 * st["peel_mids"][tier]
                 + 24 * st["peel_anchors"][tier]) / lau
    dur_s = st["ms_peel"][tier] / 1e3 / lau
    achieved = alg_bytes / dur_s / 1e9 if dur_s > 0 else 0.0
    peak, peak_kind = _peaks()
    traffic = None
    tr = NCU_TRAFFIC.get(names[tier])
    if tr and tr.get("src") == _src_digest():
        traffic = int(tr["dram_per_alg_byte"] * alg_bytes)
    gold_ok = None
    import synth
    gpath = os.path.join(ROOT, "tests", "golden", synth.CHUNG_LU_10M + ".json")
    if os.path.exists(gpath):
        gold = json.load(open(gpath))
        gold_ok = hashlib.sha256(tips.astype("<u8").tobytes()).hexdigest() == gold["tips_sha256"]

    line = {"metric": METRIC, "value": value, "unit": "wedges/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nu": nu, "nv": nv, "m": int(len(eu)), "side": "U",
                       "round_graphs": bool(args.round_graphs),
                       "P": args.P or tuned.get("P", 150), "tuning": tuned or "defaults",
                       "huc": {"mode": args.huc, "factor_1024": args.huc_factor_1024 or 8192},
                       "wedges_bup": wedges, "parallelism": "replicas" if world > 1
                       else "single", "l2": "flushed between steps (256 MiB write)"},
            "seconds_per_step": ms / 1e3,
            "bit_exact_vs_oracle": gold_ok,
            "walked_wedges_per_step": {"count": st["wedges_count"], "cd": sum(st["peel_wedges"]),
                                       "cd_without_dgm": st["wedges_cd"], "fd": st["wedges_fd"]},
            "phase_wedges_per_s": {
                "count": st["wedges_count"] / (st["ms_count"] / 1e3) if st["ms_count"] else None,
                "cd": sum(st["peel_wedges"]) / (st["ms_cd"] / 1e3) if st["ms_cd"] else None,
                "fd": st["wedges_fd"] / (st["ms_fd"] / 1e3) if st["ms_fd"] else None},
            "phase_ms": {"count": st["ms_count"], "cd": st["ms_cd"], "fd": st["ms_fd"],
                         "peel_tiers": st["ms_peel"]},
            "rounds_cd": st["rounds_cd"], "levels_fd": st["levels_fd"], "subsets": st["p_eff"],
            "fd_slowest_task": {"ms": st["ms_fd_max_subset"], "n": st["fd_max_subset_n"],
                                "levels": st["fd_max_subset_levels"]},
            "fd_heavy": {"subsets": st["fd_heavy_subsets"], "ms": st["ms_fd_heavy"],
                         "levels": st["levels_fd_heavy"]},
            "huc": {"recounts": st["huc_recounts"], "wedges": st["wedges_recount"],
                    "ms": st["ms_recount"], "cost_recount": st["cost_recount"]},
            "peel_tier_wedges": st["peel_wedges"], "peel_tier_anchors": st["peel_anchors"],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": names[tier],
                         "peak_source": peak_kind,
                         "bytes_per_launch": alg_bytes, "launch_ms": dur_s * 1e3},
            "e2e": {"value": replica_rate(wedges, world, e2e_s), "unit": "wedges/s",
                    "h2d_bytes_per_step": int(eu.nbytes + ev.nbytes),
                    "d2h_bytes_per_step": int(n_side * 8), "seconds": e2e_s,
                    "matches_device_path": e2e_ok},
            "gpu_launches": int(launches),
            "clocks": clk.summary()}
    if world == 1 and not args.no_cpu_baseline:
        cb, _ = cpu_baseline(eu, ev, nu, nv, side)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _gen_spec(spec):
    import synth
    eu, ev = synth.graph_from_spec(spec)
    return eu, ev


def _generate(specs, workers=None):
    """Draws the graphs of a batch/serving spec list in parallel host processes."""
    import multiprocessing as mp
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_gen_spec, specs, chunksize=4)


def run_batch(args):
    """Batched workload: 4,096 graphs (seed 4), U side, one packed
    decomposition versus one decomposition per graph on the same GPU."""
    import torch
    import synth
    specs = synth.batch_specs(args.batch_graphs, seed=4)
    graphs = _generate(specs)
    import paper_2010_08695_gb300 as R
    R.load()
    built = [R.Graph(eu, ev, s.nu, s.nv) for (eu, ev), s in zip(graphs, specs)]
    sides = [0] * len(built)
    torch.cuda.synchronize()
    edges = sum(g.m for g in built)
    wedges = 0
    for (eu, ev), s in zip(graphs, specs):
        dv = np.bincount(ev, minlength=s.nv).astype(np.int64)
        wedges += int((dv * (dv - 1)).sum())
    outs = R.receipt_decompose_batch(built, sides, round_graphs=args.round_graphs)  # warm-up
    torch.cuda.synchronize()
    tb = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        outs = R.receipt_decompose_batch(built, sides, outs=outs, timing=True,
                                         round_graphs=args.round_graphs)
        torch.cuda.synchronize()
        tb.append(time.perf_counter() - t0)
    batch_stats = built[0].stats()
    if args.trace:
        with open(args.trace, "w") as f:
            json.dump(built[0].trace(), f)
    alone = [torch.empty_like(o) for o in outs]
    for g, o in zip(built[:64], alone[:64]):  # warm-up
        g.tip_decompose(0, out=o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g, o in zip(built, alone):
        g.tip_decompose(0, out=o)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    same = all(torch.equal(a, b) for a, b in zip(outs, alone))
    import oracle
    sample = list(range(0, len(built), max(1, len(built) // 16)))
    oracle_ok = all(np.array_equal(R.as_u64(outs[i]), oracle.bup(graphs[i][0], graphs[i][1],
                                                                  specs[i].nu, specs[i].nv, 0)[0])
                    for i in sample)
    tbm = statistics.median(tb)
    line = {"metric": "graphs/s (batched tip decomposition)", "value": len(built) / tbm,
            "unit": "graphs/s", "n_gpus": 1, "steps": args.steps, "higher_is_better": True,
            "config": {"workload": f"{len(built)} Chung-Lu graphs, seed 4, U side",
                       "edges": edges, "wedges_bup": wedges},
            "seconds_batched": tbm, "seconds_one_graph_per_launch": t_plain,
            "graphs_per_s_one_graph_per_launch": len(built) / t_plain,
            "speedup_vs_one_graph_per_launch": t_plain / tbm,
            "wedges_per_s_batched": wedges / tbm,
            "rounds_cd": batch_stats["rounds_cd"], "subsets": batch_stats["p_eff"],
            "phase_ms": {"count": batch_stats["ms_count"], "cd": batch_stats["ms_cd"],
                         "fd": batch_stats["ms_fd"], "peel_tiers": batch_stats["ms_peel"]},
            "fd_slowest_task": {"ms": batch_stats["ms_fd_max_subset"],
                                "n": batch_stats["fd_max_subset_n"],
                                "levels": batch_stats["fd_max_subset_levels"]},
            "fd_tasks": batch_stats["fd_tasks"],
            "walked_wedges": {"count": batch_stats["wedges_count"], "cd": sum(batch_stats["peel_wedges"]),
                              "cd_without_dgm": batch_stats["wedges_cd"],
                              "fd": batch_stats["wedges_fd"]},
            "batch_equals_alone": same, "oracle_sample_ok": oracle_ok,
            "oracle_sample": len(sample)}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving workload: a bounded prefix of the seed-5 request stream
    (Poisson arrivals at 0.8x the measured one-at-a-time throughput, and a
    flood with every request at t=0), latency p50/p99 and graphs/s."""
    import torch
    import synth
    specs = synth.serve_specs(args.serve_requests, seed=5)
    graphs = _generate(specs)
    import paper_2010_08695_gb300 as R
    R.load()
    reqs = [(eu, ev, s.nu, s.nv, s.side) for (eu, ev), s in zip(graphs, specs)]
    edges = sum(len(r[0]) for r in reqs)
    # plain path: one request at a time through the host-buffer entry point
    calib = reqs[: min(len(reqs), args.serve_calib)]
    R.receipt_tip_decompose_host(*calib[0])
    t0 = time.perf_counter()
    for r in calib:
        R.receipt_tip_decompose_host(*r)
    plain_rate = len(calib) / (time.perf_counter() - t0)
    results = {}
    for mode in ("poisson", "flood"):
        sv = R.Server(max_inflight=args.serve_slots)
        arrivals = (synth.poisson_arrivals(len(reqs), 0.8 * plain_rate, seed=5)
                    if mode == "poisson" else np.zeros(len(reqs)))
        start = time.perf_counter()
        ids = []
        for r, t_arr in zip(reqs, arrivals):
            dt = start + t_arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids.append(sv.submit(*r)[0])
        outs = [sv.wait(i)[0] for i in ids]
        st = sv.stats()
        sv.close()
        results[mode] = (st, outs)
    st_p, outs_p = results["poisson"]
    st_f, outs_f = results["flood"]
    same = all(np.array_equal(a, b) for a, b in zip(outs_p, outs_f))
    alone_idx = list(range(0, len(reqs), max(1, len(reqs) // 20)))
    alone_ok = all(np.array_equal(outs_p[i], R.receipt_tip_decompose_host(*reqs[i]))
                   for i in alone_idx)
    import oracle
    small = [i for i in range(len(reqs)) if len(reqs[i][0]) <= 200000][:10]
    oracle_ok = all(np.array_equal(outs_p[i], oracle.bup(*reqs[i])[0]) for i in small)

    def pick(st):
        return {k: st[k] for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "graphs_per_s",
                                   "completed", "batches", "packed_requests", "peak_inflight",
                                   "peak_inflight_bytes")}
    line = {"metric": "graphs/s and p50/p99 latency (serving)", "value": st_p["graphs_per_s"],
            "unit": "graphs/s", "n_gpus": 1, "higher_is_better": True,
            "config": {"workload": f"first {len(reqs)} requests of the seed-5 stream",
                       "edges": edges, "slots": args.serve_slots,
                       "arrival_rate_per_s": 0.8 * plain_rate},
            "plain_one_at_a_time_graphs_per_s": plain_rate,
            "poisson": pick(st_p), "flood": pick(st_f),
            "mix_equals_alone_sample": alone_ok, "poisson_equals_flood": same,
            "oracle_sample_ok": oracle_ok, "oracle_sample": len(small)}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--trace", default=None,
                    help="write the per-round trace of the last timed step to this JSON file")
    ap.add_argument("--workload", choices=["single", "batch", "serve"], default="single",
                    help="single: the 10M-edge graph (default); batch: 4,096 graphs packed "
                         "vs one per launch; serve: the serving stream prefix")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--round-graphs", action="store_true",
                    help="run each coarse-grained round as one CUDA graph launch")
    ap.add_argument("--P", type=int, default=0,
                    help="subsets of the coarse-grained step (0: the tuned value)")
    ap.add_argument("--huc", type=int, default=0, choices=[-1, 0, 1],
                    help="recount rule (Sec. 4.1): 0 cost rule, -1 never, 1 every range")
    ap.add_argument("--huc-factor-1024", type=int, default=0,
                    help="factor of the recount rule in 1/1024 units (0: 8192)")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-calib", type=int, default=40)
    ap.add_argument("--serve-slots", type=int, default=4)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
