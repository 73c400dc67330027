"""Autotuner of the peel-update tier thresholds.

The coarse-grained peel update sends each peeled vertex (anchor) to one of
several aggregation tiers by its wedge count: a warp with a private table (at
most `warp_max_w` wedges), one CTA with the hybrid shared-memory engine over
the anchor's key window, or (more than `slice_min_w` wedges) CTAs that each
aggregate one key slice. The number of subsets P (the paper's Fig. 4 sweeps
it) and how often dynamic graph maintenance compacts the lists are tuned the
same way. The best values depend on the graph's degree distribution. `tune()` times every candidate pair on a built graph with CUDA
events and records the fastest under a shape class of the graph (powers of
two of the side sizes, the edge count and the largest degree of the other
side); `lookup()` returns the recorded thresholds for a graph of the same
class. Thresholds change speed only, never tip numbers.

The table lives in JSON: `tuned.json` next to this file (shipped, written by
`python -m paper_2010_08695_gb300.autotune` on a GB300) or the file named by
`$RECEIPT_TUNING`.
"""
from __future__ import annotations

import json
import math
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
SHIPPED = os.path.join(_HERE, "tuned.json")
WARP_MAX_W = (64, 128, 256)
SLICE_MIN_W = (49152, 98304, 196608, 1 << 30)
P_CANDIDATES = (75, 100, 150, 200, 300)
DGM_FRAC_1024 = (32, 64, 128, 256)
_lock = threading.Lock()
_table = None


def _path():
    return os.environ.get("RECEIPT_TUNING") or SHIPPED


def _load():
    global _table
    with _lock:
        if _table is None:
            try:
                with open(_path()) as f:
                    _table = json.load(f)
            except (OSError, ValueError):
                _table = {}
        return _table


def shape_class(nu: int, nv: int, m: int, side: int, max_deg_other: int) -> str:
    def b(x):
        return int(round(math.log2(max(1, x))))
    ns, no = (nu, nv) if side == 0 else (nv, nu)
    return f"s{b(ns)}-o{b(no)}-m{b(m)}-d{b(max_deg_other)}"


def lookup(key: str):
    """Thresholds recorded for a shape class, or None."""
    return _load().get(key)


def _time(graph, side, out, reps, **kw):
    import torch
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.tip_decompose(side, out=out, **kw)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(graph, side: int, key: str, reps: int = 1, save: bool = True):
    """Coordinate search on `graph`: the tier thresholds (warp_max_w,
    slice_min_w) at P = 150, then P, then the compaction trigger of dynamic
    graph maintenance. Records the fastest setting under `key` and returns
    (best, all timings in ms)."""
    import torch
    n = graph.nu if side == 0 else graph.nv
    out = torch.empty(n, dtype=torch.int64, device=graph.device)
    base = dict(P=150, dgm_frac_1024=128)
    graph.tip_decompose(side, out=out, warp_max_w=256, slice_min_w=SLICE_MIN_W[1], **base)
    times = {}
    for w in WARP_MAX_W:
        for s in SLICE_MIN_W:
            times[f"w{w},s{s},P150,f128"] = _time(graph, side, out, reps, warp_max_w=w,
                                                  slice_min_w=s, **base)
    best = min(times, key=times.get)
    w, s = (int(t[1:]) for t in best.split(",")[:2])
    for P in P_CANDIDATES:
        times[f"w{w},s{s},P{P},f128"] = _time(graph, side, out, reps, warp_max_w=w, slice_min_w=s,
                                              P=P, dgm_frac_1024=128)
    best = min(times, key=times.get)
    P = int(best.split(",")[2][1:])
    for f in DGM_FRAC_1024:
        times[f"w{w},s{s},P{P},f{f}"] = _time(graph, side, out, reps, warp_max_w=w,
                                              slice_min_w=s, P=P, dgm_frac_1024=f)
    best = min(times, key=times.get)
    w, s, P, f = (int(t[1:]) for t in best.split(","))
    rec = {"warp_max_w": w, "slice_min_w": s, "P": P, "dgm_frac_1024": f, "ms": times[best]}
    if save:
        table = dict(_load())
        table[key] = rec
        tmp = _path() + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, _path())
        with _lock:
            global _table
            _table = table
    return rec, times


def main():
    """Tunes the shape classes of the benchmark workloads and writes the table."""
    import numpy as np
    import sys
    sys.path.insert(0, os.path.dirname(_HERE))
    import synth
    import paper_2010_08695_gb300 as R
    for name in (synth.CHUNG_LU_10M,):
        eu, ev, nu, nv, side = synth.workload_graph(name)
        d_other = np.bincount(ev if side == 0 else eu, minlength=nv if side == 0 else nu)
        key = shape_class(nu, nv, len(eu), side, int(d_other.max()))
        g = R.Graph(eu, ev, nu, nv)
        rec, times = tune(g, side, key)
        print(json.dumps({"workload": name, "key": key, "best": rec, "times_ms": times}))


if __name__ == "__main__":
    main()
