#!/usr/bin/env python
"""Benchmark of RECEIPT tip decomposition on one GB300.

Headline workload: the Chung-Lu bipartite graph with |U| = 5,000,000,
|V| = 1,000,000, 100,000,000 distinct edges, exponent 2.0 on both sides
(largest expected degree 500,000 on both; drawn: 193k on U, 254k on V),
seed 3; the V side is decomposed (wedges through U, ~1.06e12 bottom-up
wedges). It is the largest single-GPU workload of the method's
configurations.

One step = one whole pass of the hot path on the device: graph build
(deduplication, degree relabelling, two-sided CSR), per-vertex butterfly
counting (Algorithm 1), coarse-grained range peeling (Algorithm 3) and
fine-grained subset peeling (Algorithm 4), from an edge list already in HBM
to tip numbers in HBM. The timed steps run without any instrumentation;
two further steps with per-tier CUDA events give the phase split and the
roofline of the dominant peel kernel.

Metric: wedges/s, where the wedge count of a step is the graph's bottom-up
peeling wedge count sum_{y in other side} d_y (d_y - 1) (the work
Algorithm 2 does; a property of the graph, the same for every
implementation), divided by the step's device time. Seconds per step, the
wedges the kernels actually walked and the roofline fraction of the
dominant kernel are reported beside it.

The same JSON line carries (N = 1, unless --no-extras): the 10M-edge
Chung-Lu workload (U side) as a secondary measurement, the 4,096-graph batch
(one packed call against one call per graph) and the first 200 requests of
the seed-5 serving stream (p50/p99 latency, graphs/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload chung-lu-5Mx1M-100M|chung-lu-1Mx200k-10M|batch|serve]

With N > 1 (torchrun, one rank per GPU) every rank decomposes its own copy of
the graph (the path has no exchange step: replicas only); the value is the
wedges of all ranks divided by the slowest rank's time.

--impl reference times the CPU oracle (test infrastructure) on the host
cores: its per-vertex butterfly count by definition (the 2-hop walk every
peeled vertex makes in Algorithm 2) over a seeded sample of the decomposed
side's vertices of the same workload, each step a bounded sample.
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
HEADLINE = "chung-lu-5Mx1M-100M"
SECONDARY = "chung-lu-1Mx200k-10M"
DESCR = {
    "chung-lu-5Mx1M-100M": "chung-lu |U|=5M |V|=1M m=100M gamma 2.0/2.0 seed 3, V side",
    "chung-lu-1Mx200k-10M": "chung-lu |U|=1M |V|=200k m=10M gamma 2.5/2.1 seed 2, U side",
    "chung-lu-2Mx400k-20M": "chung-lu |U|=2M |V|=400k m=20M gamma 2.0/2.0 seed 33, V side "
                            "(the 100M-edge graph's shape at a fifth of its size)",
}
CPU_SAMPLE_WEDGES = 2_500_000_000  # oracle walk per CPU-baseline sample (~10 s on one core)
REF_STEP_WEDGES = 800_000_000      # oracle walk per reference-arm step (~3-4 s)
SERVE_PREFIX = 200

# DRAM traffic of a peel kernel from one ncu capture, as DRAM bytes per
# algorithmic byte of the captured launch (scaled to the average launch of
# the step), keyed by kernel name; valid only while the peel kernels'
# sources (PEEL_SOURCES) hash to the recorded digest.
NCU_TRAFFIC = {
    # rounds 134-138 of the 100M-edge decomposition (the heaviest sliced
    # round and the next four): 4.032 GB of DRAM traffic for 76.97 GB of
    # algorithmic bytes
    "k_cd_update_slice": {"src": "f2b774bbdaf08fc7", "dram_per_alg_byte": 0.05238},
}

PEEL_TIERS = ["k_cd_update_warp", "k_cd_update_cta", "k_cd_update_global", "k_cd_update_slice",
              "k_cd_update_dense"]


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


def load_workload(name):
    import synth
    eu, ev, nu, nv, side = synth.workload_graph(name)
    d = np.bincount(ev if side == 0 else eu, minlength=nv if side == 0 else nu).astype(np.int64)
    wedges = int((d * (d - 1)).sum())
    return eu, ev, nu, nv, side, wedges


def roofline(st, peak, peak_kind):
    """Roofline of the peel tier with the most device time in the
    instrumented step(s): algorithmic bytes per launch (4 B per wedge walked,
    16 B per middle-vertex visit, 16 B per support atomic, 24 B per anchor)
    over the tier's average launch time."""
    tier = max(range(5), key=lambda t: st["ms_peel"][t])
    lau = max(1, st["peel_launches"][tier])
    alg_bytes = (4 * st["peel_wedges"][tier] + 16 * st["peel_mids"][tier]
                 + 16 * st["peel_pairs"][tier] + 24 * st["peel_anchors"][tier]) / lau
    dur_s = st["ms_peel"][tier] / 1e3 / lau
    achieved = alg_bytes / dur_s / 1e9 if dur_s > 0 else 0.0
    traffic = None
    tr = NCU_TRAFFIC.get(PEEL_TIERS[tier])
    if tr and tr.get("src") == _src_digest():
        traffic = int(tr["dram_per_alg_byte"] * alg_bytes)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": PEEL_TIERS[tier],
            "peak_source": peak_kind, "bytes_per_launch": alg_bytes, "launch_ms": dur_s * 1e3,
            "launches": lau, "bytes_model": "4 B/wedge + 16 B/mid + 16 B/pair + 24 B/anchor"}


def _mean_stats(stats):
    """Field-wise mean of instrumented steps' stats (lists element-wise)."""
    out = {}
    for k in stats[0]:
        v = [s[k] for s in stats]
        if isinstance(v[0], list):
            out[k] = [sum(x) / len(x) for x in zip(*v)]
        else:
            out[k] = sum(v) / len(v)
    return out


def measure_graph(R, name, args, dist=None, world=1, local=0, clocks=True, e2e=True,
                  roofline_steps=2):
    """Times `steps` uninstrumented device steps of the named workload (after
    `warmup`), then `roofline_steps` instrumented ones, then the end-to-end
    leg through the host-buffer entry point. Returns the measurement dict."""
    import torch
    eu, ev, nu, nv, side, wedges = load_workload(name)
    n_side = nu if side == 0 else nv
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    eu_d = torch.from_numpy(eu).to(dev)
    ev_d = torch.from_numpy(ev).to(dev)
    tip = torch.empty(n_side, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    from paper_2010_08695_gb300 import autotune
    g0 = R.Graph(eu_d, ev_d, nu, nv, stream=stream)
    tuned = autotune.lookup(g0.shape_class(side)) or {}
    g0.close()
    P = args.P or tuned.get("P", 150)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    trace = []

    def step(timing):
        g = R.Graph(eu_d, ev_d, nu, nv, stream=stream)
        g.tip_decompose(side, P=P, timing=timing, out=tip, stream=stream,
                        round_graphs=args.round_graphs, huc=args.huc,
                        huc_factor_1024=args.huc_factor_1024)
        st = g.stats()
        if timing and args.trace:
            trace[:] = g.trace()
        g.close()
        return st

    for _ in range(max(3, args.warmup)):
        step(False)
    barrier()
    times, plain = [], []
    launches0 = R.receipt_kernel_launches()

    class _Null:
        def __enter__(self):
            return self

        def __exit__(self, *a):
            pass

        def summary(self):
            return None
    with (ClockSampler(local) if clocks else _Null()) as clk:
        barrier()
        for _ in range(args.steps):
            flush.fill_(1.0)  # evicts L2 between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plain.append(step(False))
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        barrier()
    launches = R.receipt_kernel_launches() - launches0
    ms = max_over_ranks(statistics.mean(times), dist, dev)
    tips = R.as_u64(tip)
    # instrumented steps: phase split, per-tier counters and device time
    inst, inst_ms = [], []
    for _ in range(roofline_steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst.append(step(True))
        e1.record(stream)
        e1.synchronize()
        inst_ms.append(e0.elapsed_time(e1))
    if not inst:  # no instrumented step: counters of one more plain-timing step
        inst.append(step(True))
        inst_ms.append(float("nan"))
    st = _mean_stats(inst)
    last = inst[-1]
    peak, peak_kind = _peaks()
    out = {
        "workload": DESCR.get(name, name), "nu": nu, "nv": nv, "m": int(len(eu)),
        "side": "U" if side == 0 else "V", "wedges_bup": wedges, "P": P,
        "tuning": tuned or "defaults", "ms_per_step": ms, "value": replica_rate(wedges, world, ms / 1e3),
        "step_ms_all": times, "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "instrumented_step_ms": statistics.mean(inst_ms),
        "walked_wedges_per_step": {"count": last["wedges_count"], "cd": sum(last["peel_wedges"]),
                                   "cd_without_dgm": last["wedges_cd"], "fd": last["wedges_fd"]},
        "phase_ms": {"count": st["ms_count"], "cd": st["ms_cd"], "fd": st["ms_fd"],
                     "peel_tiers": st["ms_peel"],
                     "cd_outside_tiers": st["ms_cd"] - sum(st["ms_peel"])},
        # the timed (uninstrumented) steps' own phase split: rounds run
        # device-driven, tiers on forked streams
        "phase_ms_timed_steps": {k: statistics.mean(p[f"ms_{k}"] for p in plain)
                                 for k in ("count", "cd", "fd")} if plain else None,
        "phase_wedges_per_s": {
            "count": last["wedges_count"] / (st["ms_count"] / 1e3) if st["ms_count"] else None,
            "cd": sum(last["peel_wedges"]) / (st["ms_cd"] / 1e3) if st["ms_cd"] else None,
            "fd": last["wedges_fd"] / (st["ms_fd"] / 1e3) if st["ms_fd"] else None},
        "rounds_cd": last["rounds_cd"], "levels_fd": last["levels_fd"], "subsets": last["p_eff"],
        "fd_slowest_task": {"ms": st["ms_fd_max_subset"], "n": last["fd_max_subset_n"],
                            "levels": last["fd_max_subset_levels"]},
        "fd_heavy": {"subsets": last["fd_heavy_subsets"], "ms": st["ms_fd_heavy"],
                     "levels": last["levels_fd_heavy"]},
        "huc": {"mode": args.huc, "recounts": last["huc_recounts"],
                "wedges": last["wedges_recount"], "ms": st["ms_recount"],
                "cost_recount": last["cost_recount"]},
        "peel_tier_wedges": last["peel_wedges"], "peel_tier_anchors": last["peel_anchors"],
        "peel_tier_pairs": last["peel_pairs"], "peel_tier_mids": last["peel_mids"],
        "roofline": roofline(st, peak, peak_kind),
    }
    import synth
    gpath = os.path.join(ROOT, "tests", "golden", name + ".json")
    out["bit_exact_vs_oracle"] = None
    if os.path.exists(gpath):
        gold = json.load(open(gpath))
        if "tips_sha256" in gold and synth.edges_sha256(eu, ev) == gold["edges_sha256"]:
            out["bit_exact_vs_oracle"] = (
                hashlib.sha256(tips.astype("<u8").tobytes()).hexdigest() == gold["tips_sha256"])
    if args.trace and trace:
        with open(args.trace, "w") as f:
            json.dump(trace, f)
    del flush
    if e2e:
        # end to end through the C ABI with host buffers: H2D of the edges,
        # build, decomposition, D2H of the tips, with the step's options
        e2e_opt = {k: tuned.get(k, 0) for k in ("warp_max_w", "slice_min_w", "dgm_frac_1024",
                                                 "slice_ctas", "slice_fetch")}
        e2e_opt["range_max_n"] = R._tuned_cap(tuned, P) if tuned else 0
        e2e_opt.update(huc=args.huc, huc_factor_1024=args.huc_factor_1024,
                       round_graphs=args.round_graphs)
        eu_h = torch.from_numpy(eu).pin_memory().numpy()
        ev_h = torch.from_numpy(ev).pin_memory().numpy()
        tip_h = torch.empty(n_side, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
        R.receipt_tip_decompose_host(eu_h, ev_h, nu, nv, side, P=P, out=tip_h, **e2e_opt)
        e2e_t = []
        for _ in range(max(1, min(args.steps, 3))):
            barrier()
            t0 = time.perf_counter()
            R.receipt_tip_decompose_host(eu_h, ev_h, nu, nv, side, P=P, out=tip_h, **e2e_opt)
            e2e_t.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(statistics.mean(e2e_t), dist, dev)
        out["e2e"] = {"value": replica_rate(wedges, world, e2e_s), "unit": "wedges/s",
                      "h2d_bytes_per_step": int(eu.nbytes + ev.nbytes),
                      "d2h_bytes_per_step": int(n_side * 8), "seconds": e2e_s,
                      "matches_device_path": bool(np.array_equal(tip_h, tips))}
    return out, (eu, ev, nu, nv, side)


def _vertex_sample(eu, ev, nu, nv, side, budget, seed):
    """Seeded random vertices of the decomposed side whose 2-hop walks
    (sum over y in N_x of d_y) add up to about `budget` entries."""
    a, b, nb = (eu, ev, nv) if side == 0 else (ev, eu, nu)
    na = nu if side == 0 else nv
    d_o = np.bincount(b, minlength=nb).astype(np.float64)
    walk = np.bincount(a, weights=d_o[b], minlength=na)
    order = np.random.default_rng(seed).permutation(na)
    k = int(np.searchsorted(np.cumsum(walk[order]), budget)) + 1
    return order[:k].astype(np.int32)


def cpu_oracle_rate(graph, eu, ev, nu, nv, side, budget, seed):
    """Wedges/s of the oracle's per-vertex count by definition over a seeded
    vertex sample (one core; adjacency built beforehand)."""
    xs = _vertex_sample(eu, ev, nu, nv, side, budget, seed)
    t0 = time.perf_counter()
    _, walked = graph.count_vertex(side, xs)
    dt = time.perf_counter() - t0
    return walked / dt, walked, dt, len(xs)


def cpu_baseline(eu, ev, nu, nv, side, name):
    import oracle
    t0 = time.perf_counter()
    g = oracle.Graph(eu, ev, nu, nv)
    t_build = time.perf_counter() - t0
    rate, walked, dt, k = cpu_oracle_rate(g, eu, ev, nu, nv, side, CPU_SAMPLE_WEDGES, 1)
    g.close()
    return {"value": rate, "unit": "wedges/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle per-vertex butterfly count by definition (the 2-hop walk of "
                       f"Algorithm 2's update) of {k} seeded random {('U', 'V')[side]} vertices "
                       f"of {name}: {walked} wedges in {dt:.1f} s on one core (adjacency built "
                       f"once beforehand in {t_build:.1f} s, not in the rate)")}


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    import oracle
    name = args.workload if args.workload in DESCR else HEADLINE
    eu, ev, nu, nv, side, wedges = load_workload(name)
    g = oracle.Graph(eu, ev, nu, nv)
    for i in range(args.warmup):
        cpu_oracle_rate(g, eu, ev, nu, nv, side, REF_STEP_WEDGES // 8, 1000 + i)
    rates, secs, walks = [], [], []
    for i in range(args.steps):
        r, w, dt, _ = cpu_oracle_rate(g, eu, ev, nu, nv, side, REF_STEP_WEDGES, i)
        rates.append(r)
        secs.append(dt)
        walks.append(w)
    g.close()
    value = sum(walks) / sum(secs)
    sample = (f"oracle per-vertex butterfly count by definition over a seeded sample of "
              f"{('U', 'V')[side]} vertices of {name}, ~{REF_STEP_WEDGES} wedges per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "wedges/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": DESCR[name], "nu": nu, "nv": nv, "m": int(len(eu)),
                       "side": "U" if side == 0 else "V", "wedges_bup": wedges,
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": "wedges/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "wedges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
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


def batch_leg(R, args):
    """4,096 graphs (seed 4), U side: one packed decomposition versus one
    decomposition per graph on the same GPU."""
    import torch
    import synth
    specs = synth.batch_specs(args.batch_graphs, seed=4)
    graphs = _generate(specs)
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
    for _ in range(3):
        t0 = time.perf_counter()
        outs = R.receipt_decompose_batch(built, sides, outs=outs, round_graphs=args.round_graphs)
        torch.cuda.synchronize()
        tb.append(time.perf_counter() - t0)
    # the same with every coarse-grained round as one CUDA graph launch
    tg = []
    outs_g = R.receipt_decompose_batch(built, sides, round_graphs=True)
    torch.cuda.synchronize()
    for _ in range(3):
        t0 = time.perf_counter()
        outs_g = R.receipt_decompose_batch(built, sides, outs=outs_g, round_graphs=True)
        torch.cuda.synchronize()
        tg.append(time.perf_counter() - t0)
    same_g = all(torch.equal(a, b) for a, b in zip(outs, outs_g))
    R.receipt_decompose_batch(built, sides, outs=outs, timing=True, round_graphs=args.round_graphs)
    bs = built[0].stats()
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
    tbm = statistics.median(tb)
    return {"workload": f"{len(built)} Chung-Lu graphs, seed 4, U side", "edges": edges,
            "wedges_bup": wedges, "graphs_per_s": len(built) / tbm, "seconds_batched": tbm,
            "seconds_one_graph_per_launch": t_plain,
            "graphs_per_s_one_graph_per_launch": len(built) / t_plain,
            "speedup_vs_one_graph_per_launch": t_plain / tbm,
            "wedges_per_s_batched": wedges / tbm,
            "graphs_per_s_rounds_as_cuda_graphs": len(built) / statistics.median(tg),
            "rounds_as_cuda_graphs_equal": same_g, "rounds_cd": bs["rounds_cd"],
            "subsets": bs["p_eff"], "fd_tasks": bs["fd_tasks"],
            "phase_ms": {"count": bs["ms_count"], "cd": bs["ms_cd"], "fd": bs["ms_fd"],
                         "peel_tiers": bs["ms_peel"]},
            "fd_slowest_task": {"ms": bs["ms_fd_max_subset"], "n": bs["fd_max_subset_n"],
                                "levels": bs["fd_max_subset_levels"]},
            "batch_equals_alone": same}


def serve_leg(R, args):
    """The first `serve_requests` requests of the seed-5 serving stream:
    Poisson arrivals at 0.8x the measured one-at-a-time throughput, and a
    flood with every request at t = 0; latency p50/p99 and graphs/s."""
    import synth
    specs = synth.serve_specs(args.serve_requests, seed=5)
    graphs = _generate(specs)
    reqs = [(eu, ev, s.nu, s.nv, s.side) for (eu, ev), s in zip(graphs, specs)]
    edges = sum(len(r[0]) for r in reqs)
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

    def pick(st):
        return {k: st[k] for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "graphs_per_s",
                                   "completed", "batches", "packed_requests", "peak_inflight",
                                   "peak_inflight_bytes")}
    return {"workload": f"first {len(reqs)} requests of the seed-5 stream", "edges": edges,
            "slots": args.serve_slots, "arrival_rate_per_s": 0.8 * plain_rate,
            "plain_one_at_a_time_graphs_per_s": plain_rate,
            "poisson": pick(st_p), "flood": pick(st_f),
            "mix_equals_alone_sample": alone_ok, "poisson_equals_flood": same}


def run_single(args):
    """One decomposition of a single-graph workload (for profiler captures):
    prints its seconds and, with --trace, writes its per-round trace."""
    import torch
    import paper_2010_08695_gb300 as R
    torch.cuda.set_device(_rank_env()[2])
    R.load()
    eu, ev, nu, nv, side, wedges = load_workload(args.workload)
    g = R.Graph(eu, ev, nu, nv)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tip = g.tip_decompose(side, P=args.P, timing=bool(args.trace), fd_heavy_w=args.fd_heavy_w)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st = g.stats()
    if args.trace:
        with open(args.trace, "w") as f:
            json.dump(g.trace(), f)
    print(json.dumps({"workload": args.workload, "seconds": dt, "rounds_cd": st["rounds_cd"],
                      "peel_wedges": st["peel_wedges"], "peel_pairs": st["peel_pairs"],
                      "tips_sha256": hashlib.sha256(R.as_u64(tip).astype("<u8").tobytes())
                      .hexdigest()}), flush=True)
    return 0


def run_experiments(args):
    """The paper's experiments on the synthetic workloads (Sec. 5): a sweep of
    P (Fig. 4), the ablation of the recount (Sec. 4.1) and of dynamic graph
    maintenance (Sec. 4.2) (Figs. 5-6: RECEIPT, without the recount, without
    both) and the phase breakup (Sec. 5.2.3), one instrumented step per
    setting after a warm-up step, tip numbers checked against the first
    setting's. Writes one JSON record per workload to args.experiments."""
    import torch
    import paper_2010_08695_gb300 as R
    torch.cuda.set_device(_rank_env()[2])
    R.load()
    names = [args.workload] if args.workload in DESCR else [SECONDARY, HEADLINE]
    out = {}
    for name in names:
        eu, ev, nu, nv, side, wedges = load_workload(name)
        dev = torch.device("cuda", torch.cuda.current_device())
        eu_d = torch.from_numpy(eu).to(dev)
        ev_d = torch.from_numpy(ev).to(dev)
        n_side = nu if side == 0 else nv
        tip = torch.empty(n_side, dtype=torch.int64, device=dev)
        ref = None
        # few subsets: P = 4 on the 10M-edge graph; on the 100M-edge graph a
        # subset of P = 4 takes minutes to peel exactly (P = 25 instead). The
        # slow small-P settings run last.
        few = 4 if name == SECONDARY else 25
        ps = (50, 100, 150, 300, 600, 25, 4) if name == SECONDARY else \
            (100, 150, 200, 300, 600, 50, 25)
        settings = [("P", {"P": p}) for p in ps]
        settings += [("receipt", {"P": 150}),
                     ("receipt-paper-huc-factor", {"P": 150, "huc_factor_1024": 1024}),
                     ("receipt-no-huc", {"P": 150, "huc": -1}),
                     ("receipt-no-huc-no-dgm", {"P": 150, "huc": -1, "dgm": False}),
                     (f"receipt-P{few}", {"P": few}),
                     (f"receipt-P{few}-paper-huc-factor", {"P": few, "huc_factor_1024": 1024}),
                     (f"receipt-P{few}-no-huc", {"P": few, "huc": -1}),
                     (f"receipt-P{few}-no-huc-no-dgm", {"P": few, "huc": -1, "dgm": False})]
        recs = []
        for label, kw in settings:
            rec = {"setting": label, **{k: v for k, v in kw.items()}}
            for t in (False, True):
                g = R.Graph(eu_d, ev_d, nu, nv)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                g.tip_decompose(side, out=tip, timing=t, **kw)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                st = g.stats()
                g.close()
            tips = R.as_u64(tip).copy()
            if ref is None:
                ref = tips
            rec.update({"seconds": dt, "ms_count": st["ms_count"], "ms_cd": st["ms_cd"],
                        "ms_fd": st["ms_fd"], "rounds_cd": st["rounds_cd"],
                        "levels_fd": st["levels_fd"], "subsets": st["p_eff"],
                        "wedges_count": st["wedges_count"],
                        "wedges_cd_walked": sum(st["peel_wedges"]),
                        "wedges_cd_without_dgm": st["wedges_cd"], "wedges_fd": st["wedges_fd"],
                        "recounts": st["huc_recounts"], "wedges_recount": st["wedges_recount"],
                        "ms_recount": st["ms_recount"], "fd_slowest_task_ms": st["ms_fd_max_subset"],
                        "fd_heavy_subsets": st["fd_heavy_subsets"],
                        "same_tips_as_first": bool(np.array_equal(tips, ref))})
            recs.append(rec)
            print(json.dumps({"workload": name, **rec}), flush=True)
        out[name] = {"workload": DESCR[name], "wedges_bup": wedges, "records": recs,
                     "note": "seconds: one step with per-phase CUDA events, after an "
                             "uninstrumented warm-up step of the same setting"}
        with open(args.experiments, "w") as f:  # after each workload
            json.dump(out, f, indent=1)
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
    name = args.workload
    main, graph = measure_graph(R, name, args, dist, world, local,
                                roofline_steps=args.roofline_steps)
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": main["value"], "unit": "wedges/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": main["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": main["workload"], "nu": main["nu"], "nv": main["nv"],
                       "m": main["m"], "side": main["side"], "wedges_bup": main["wedges_bup"],
                       "P": main["P"], "tuning": main["tuning"],
                       "round_graphs": bool(args.round_graphs),
                       "huc": {"mode": args.huc, "factor_1024": args.huc_factor_1024 or 8192},
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed between steps (256 MiB write)",
                       "timed_steps": "uninstrumented; phase split and roofline from 2 "
                                      "further steps with per-tier CUDA events"},
            "seconds_per_step": main["ms_per_step"] / 1e3,
            "bit_exact_vs_oracle": main["bit_exact_vs_oracle"],
            "roofline": main["roofline"], "e2e": main["e2e"],
            "gpu_launches": main["gpu_launches"], "clocks": main["clocks"]}
    for k in ("step_ms_all", "instrumented_step_ms", "walked_wedges_per_step", "phase_ms",
              "phase_ms_timed_steps",
              "phase_wedges_per_s", "rounds_cd", "levels_fd", "subsets", "fd_slowest_task",
              "fd_heavy", "huc", "peel_tier_wedges", "peel_tier_anchors", "peel_tier_pairs",
              "peel_tier_mids"):
        line[k] = main[k]
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(*graph, name)
    if world == 1 and not args.no_extras:
        if name != SECONDARY:
            sec_args = argparse.Namespace(**vars(args))
            sec_args.steps, sec_args.warmup, sec_args.P, sec_args.trace = 5, 3, 0, None
            sec, _ = measure_graph(R, SECONDARY, sec_args, clocks=False, roofline_steps=1)
            for k in ("step_ms_all", "clocks", "peel_tier_mids"):
                sec.pop(k, None)
            line["secondary"] = sec
        line["batch"] = batch_leg(R, args)
        line["serve"] = serve_leg(R, args)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the secondary workload, the batch and the serving legs")
    ap.add_argument("--roofline-steps", type=int, default=2,
                    help="instrumented steps after the timed ones (phase split, roofline)")
    ap.add_argument("--trace", default=None,
                    help="write the per-round trace of the last instrumented step to this file")
    ap.add_argument("--workload", default=HEADLINE,
                    choices=[HEADLINE, SECONDARY, "chung-lu-2Mx400k-20M", "batch", "serve"],
                    help="single graph (default: the 100M-edge graph); batch: 4,096 graphs "
                         "packed vs one per launch; serve: the serving stream prefix")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--round-graphs", action="store_true",
                    help="run each coarse-grained round as one CUDA graph launch")
    ap.add_argument("--P", type=int, default=0,
                    help="subsets of the coarse-grained step (0: the tuned value)")
    ap.add_argument("--huc", type=int, default=0, choices=[-1, 0, 1],
                    help="recount rule (Sec. 4.1): 0 cost rule, -1 never, 1 every range")
    ap.add_argument("--huc-factor-1024", type=int, default=0,
                    help="factor of the recount rule in 1/1024 units (0: 8192)")
    ap.add_argument("--fd-heavy-w", type=int, default=0,
                    help="--single: heavy-task threshold of the fine-grained step (0 automatic, "
                         "-1 never)")
    ap.add_argument("--single", action="store_true",
                    help="one decomposition of the workload and nothing else (profiling runs)")
    ap.add_argument("--experiments", default=None,
                    help="run the P sweep and the recount/maintenance ablation and write "
                         "them to this JSON file (instead of the benchmark)")
    ap.add_argument("--serve-requests", type=int, default=SERVE_PREFIX)
    ap.add_argument("--serve-calib", type=int, default=40)
    ap.add_argument("--serve-slots", type=int, default=4)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.experiments:
        return run_experiments(args)
    if args.single:
        return run_single(args)
    if args.workload in ("batch", "serve"):
        import torch
        torch.cuda.set_device(_rank_env()[2])
        import paper_2010_08695_gb300 as R
        R.load()
        leg = batch_leg(R, args) if args.workload == "batch" else serve_leg(R, args)
        print(json.dumps(leg), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
