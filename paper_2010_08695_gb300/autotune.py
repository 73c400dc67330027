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
WARP_MAX_W = (256, 128, 64)
SLICE_MIN_W = (49152, 98304, 196608, 1 << 30)
P_CANDIDATES = (150, 100, 200, 300)
DGM_FRAC_1024 = (128, 64, 32)
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


def _time(run, reps, **kw):
    import torch
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        run(**kw)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def knobs(n: int):
    """Candidate values of every tuned option, in search order: the sliced
    tier's shape and its items per fetch, the tier thresholds (which anchors, by walk size, take the
    warp table, the shared-memory hybrid or the key slices), P, the vertex
    cap of a range (absolute; -1 none, 0 = 2 n / P) and the compaction
    trigger of dynamic graph maintenance."""
    return [("slice_ctas", (4, 2, 1)),
            ("slice_fetch", (1, 2, 4)),
            ("warp_max_w", WARP_MAX_W),
            ("slice_min_w", SLICE_MIN_W),
            ("P", P_CANDIDATES),
            ("range_max_n", (0, -1, max(1, n // 150), max(1, 4 * n // 150))),
            ("dgm_frac_1024", DGM_FRAC_1024)]


def search(run, n: int, reps: int = 1, time_fn=None):
    """Coordinate search: every knob in turn over its candidates with the
    others at their best so far. `run(**options)` decomposes once;
    `time_fn(run, reps, **options)` times it (default: CUDA events, best of
    `reps`). Returns (best options with their time in ms, all timings)."""
    _time_fn = time_fn or _time
    cur = {"slice_ctas": 4, "slice_fetch": 1, "warp_max_w": 256, "slice_min_w": SLICE_MIN_W[0],
           "P": 150, "range_max_n": 0, "dgm_frac_1024": 128}
    run(**cur)  # warm-up
    times = {}

    def key(o):
        return ",".join(f"{k}={o[k]}" for k in sorted(o))
    best_ms = _time_fn(run, reps, **cur)
    times[key(cur)] = best_ms
    for name, cands in knobs(n):
        for v in cands:
            o = dict(cur, **{name: v})
            k = key(o)
            if k not in times:
                times[k] = _time_fn(run, reps, **o)
            if times[k] < best_ms:
                best_ms, cur = times[k], o
    return dict(cur, ms=best_ms), times


def _save(key: str, rec: dict):
    table = dict(_load())
    table[key] = rec
    tmp = _path() + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, _path())
    with _lock:
        global _table
        _table = table


def tune(graph, side: int, key: str, reps: int = 1, save: bool = True):
    """Tunes the options of one graph's decomposition and records the best
    under `key`. Returns (best, all timings in ms)."""
    import torch
    n = graph.nu if side == 0 else graph.nv
    out = torch.empty(n, dtype=torch.int64, device=graph.device)
    rec, times = search(lambda **o: graph.tip_decompose(side, out=out, **o), n, reps)
    if save:
        _save(key, rec)
    return rec, times


def batch_shape_class(graphs, sides) -> str:
    """Shape class of the disjoint union a batch decomposes."""
    ns = sum(g.nu if s == 0 else g.nv for g, s in zip(graphs, sides))
    no = sum(g.nv if s == 0 else g.nu for g, s in zip(graphs, sides))
    m = sum(g.m for g in graphs)
    d = max((g.max_degree[1 - s] for g, s in zip(graphs, sides)), default=0)
    return "batch-" + shape_class(ns, no, m, 0, d)


def tune_batch(graphs, sides, reps: int = 1, save: bool = True):
    """Tunes the options of one packed decomposition of `graphs` and records
    them under the union's shape class."""
    from . import receipt_decompose_batch
    key = batch_shape_class(graphs, sides)
    n = sum(g.nu if s == 0 else g.nv for g, s in zip(graphs, sides))
    outs = receipt_decompose_batch(graphs, sides, tuned=False)
    rec, times = search(lambda **o: receipt_decompose_batch(graphs, sides, outs=outs, tuned=False,
                                                            **o), n, reps)
    if save:
        _save(key, rec)
    return key, rec, times


def main():
    """Tunes the shape classes of the benchmark workloads and writes the table."""
    import numpy as np
    import sys
    sys.path.insert(0, os.path.dirname(_HERE))
    import synth
    import paper_2010_08695_gb300 as R
    R.load()
    names = sys.argv[1:] or [synth.CHUNG_LU_100M, synth.CHUNG_LU_10M, "batch"]
    for name in names:
        if name == "batch":
            specs = synth.batch_specs(4096, seed=4)
            built = [R.Graph(*synth.graph_from_spec(sp), sp.nu, sp.nv) for sp in specs]
            key, rec, times = tune_batch(built, [0] * len(built))
        else:
            eu, ev, nu, nv, side = synth.workload_graph(name)
            d_other = np.bincount(ev if side == 0 else eu, minlength=nv if side == 0 else nu)
            key = shape_class(nu, nv, len(eu), side, int(d_other.max()))
            g = R.Graph(eu, ev, nu, nv)
            rec, times = tune(g, side, key)
        print(json.dumps({"workload": name, "key": key, "best": rec, "times_ms": times}), flush=True)


if __name__ == "__main__":
    main()
