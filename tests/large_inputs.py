"""Host-side inputs of the full-size parity tests.

Draws the graphs of a list of seeded specs (the batched and the serving
workloads) in spawned worker processes and, for every graph whose bottom-up
peeling wedge count sum_{y in other side} d_y (d_y - 1) is at most a bound,
runs the CPU oracle's sequential peel (Algorithm 2) on it in the same
worker, one OpenMP thread per worker. Nothing here touches the CUDA library:
the pool is started with `spawn`, so it is safe after the test process has
initialised CUDA.
"""
from __future__ import annotations

import os

import numpy as np


def _init_worker():
    # one thread per worker process: the pool already uses every core
    os.environ["OMP_NUM_THREADS"] = "1"


def bup_wedges(eu, ev, nu, nv, side):
    """sum over the other side of d(d - 1): the wedges bottom-up peeling walks."""
    d = np.bincount(ev if side == 0 else eu, minlength=nv if side == 0 else nu).astype(np.int64)
    return int((d * (d - 1)).sum())


def draw_one(item):
    """(spec, wedge_bound) -> (eu, ev, oracle tips or None, bup wedges)."""
    spec, bound = item
    import synth
    eu, ev = synth.graph_from_spec(spec)
    w = bup_wedges(eu, ev, spec.nu, spec.nv, spec.side)
    tips = None
    if bound is not None and w <= bound:
        import oracle
        tips = oracle.bup(eu, ev, spec.nu, spec.nv, spec.side)[0]
    return eu, ev, tips, w


def draw_all(specs, wedge_bound=None, chunksize=1):
    """Draws every spec's graph (and its oracle tips within `wedge_bound`;
    None = no oracle) in a spawned pool of up to 16 processes."""
    import multiprocessing as mp
    workers = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers, initializer=_init_worker) as pool:
        return pool.map(draw_one, [(s, wedge_bound) for s in specs], chunksize=chunksize)
