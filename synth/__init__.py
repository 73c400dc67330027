"""Seeded synthetic bipartite graphs: the inputs shared by the CUDA path, the
CPU oracle, the tests and the benchmark.

This module only draws edge lists. It holds none of the tip-decomposition
arithmetic (no butterfly counts, no supports, no peeling), so that the oracle
and the CUDA library can both read its output without sharing any of the
method's code.

Graphs are returned as two ``int32`` numpy arrays ``(eu, ev)`` of distinct
edges, ``eu`` in ``[0, nu)`` and ``ev`` in ``[0, nv)``, in the order in which
each distinct edge was first drawn.

Workloads (stand-ins for the KONECT bipartite datasets of the paper's
Table 2, which are heavy-tailed with hubs and average degrees of 5-118):

* ``er``       -- uniform random bipartite graph without replacement;
* ``chung_lu`` -- power-law expected degrees ``w_i ~ (i + i0)^(-1/(gamma-1))``
  on each side, expected degrees capped at the other side's size, endpoints
  drawn independently by inverse CDF, duplicates rejected and re-drawn until
  exactly ``m`` distinct edges exist;
* ``batch_specs`` / ``serve_specs`` -- the per-graph size recipes of the
  batched and the serving workloads.
"""
from __future__ import annotations

import hashlib
import math
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "er", "chung_lu", "chung_lu_i0_for_max", "edges_sha256", "workload_graph",
    "GraphSpec", "batch_specs", "serve_specs", "graph_from_spec", "WORKLOADS",
    "ER_20K", "CHUNG_LU_10M", "CHUNG_LU_100M", "CHUNG_LU_20M",
    "random_small", "complete_bipartite",
]


def edges_sha256(eu: np.ndarray, ev: np.ndarray) -> str:
    """SHA-256 of the little-endian int32 edge arrays (eu bytes then ev bytes)."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(eu, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(ev, dtype="<i4").tobytes())
    return h.hexdigest()


def er(nu: int, nv: int, m: int, seed: int):
    """Uniform bipartite graph: ``m`` distinct cells of the ``nu x nv`` grid."""
    rng = np.random.default_rng(seed)
    k = rng.choice(nu * nv, m, replace=False)
    return (k // nv).astype(np.int32), (k % nv).astype(np.int32)


def _probs(n: int, gamma: float, i0: float, m: int, cap: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    w = (i + i0) ** (-1.0 / (gamma - 1.0))
    d = m * w / w.sum()
    d = np.minimum(d, float(cap))
    return d / d.sum()


def chung_lu_i0_for_max(n: int, gamma: float, m: int, dmax: float) -> float:
    """Offset ``i0`` for which the largest expected degree ``m * p_0`` is ``dmax``
    (bisection on a log scale; the maximum falls monotonically as ``i0`` grows)."""
    def top(i0):
        i = np.arange(n, dtype=np.float64)
        w = (i + i0) ** (-1.0 / (gamma - 1.0))
        return m * w[0] / w.sum()
    lo, hi = 1e-6, 1e9
    if top(hi) > dmax:
        return hi
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if top(mid) > dmax:
            lo = mid
        else:
            hi = mid
        if hi / lo < 1 + 1e-12:
            break
    return hi


# Above this many draws the inverse-CDF search and the distinct-edge
# bookkeeping of ``chung_lu`` run on torch's multi-threaded CPU sort and
# search (exact comparisons: the same results as numpy's).
_TORCH_MIN_DRAWS = 1 << 20


def _draw(cdf: np.ndarray, rng: np.random.Generator, k: int) -> np.ndarray:
    r = rng.random(k)
    if k >= _TORCH_MIN_DRAWS:
        import torch
        idx = torch.searchsorted(torch.from_numpy(cdf), torch.from_numpy(r), right=True).numpy()
    else:
        idx = np.searchsorted(cdf, r, side="right")
    return np.minimum(idx, len(cdf) - 1).astype(np.int64)


def _first_new(keys_sorted, cand):
    """Positions (ascending) of the first occurrence of every value of `cand`
    that is absent from all the sorted arrays in `keys_sorted`."""
    if len(cand) >= _TORCH_MIN_DRAWS:
        import torch
        c = torch.from_numpy(cand)
        fresh = torch.ones(len(c), dtype=torch.bool)
        for ks in keys_sorted:
            if len(ks) == 0:
                continue
            t = torch.from_numpy(ks)
            pos = torch.clamp_max(torch.searchsorted(t, c), len(t) - 1)
            fresh &= t[pos] != c
        idx = torch.nonzero(fresh).flatten()
        sk, perm = torch.sort(c[idx], stable=True)
        first = torch.ones(len(sk), dtype=torch.bool)
        first[1:] = sk[1:] != sk[:-1]
        out, _ = torch.sort(idx[perm[first]])
        return out.numpy()
    fresh = np.ones(len(cand), dtype=bool)
    for ks in keys_sorted:
        if len(ks) == 0:
            continue
        pos = np.minimum(np.searchsorted(ks, cand), len(ks) - 1)
        fresh &= ks[pos] != cand
    idx = np.nonzero(fresh)[0]
    _, first = np.unique(cand[idx], return_index=True)
    return np.sort(idx[first])


def chung_lu(nu: int, nv: int, m: int, gamma_u: float, gamma_v: float,
             seed: int, i0_u: float = 1.0, i0_v: float = 1.0):
    """Chung-Lu bipartite graph with exactly ``m`` distinct edges.

    Rounds of independent endpoint draws (inverse CDF) continue until ``m``
    distinct edges exist; the graph is the first ``m`` distinct edges in draw
    order. Each round only checks its own draws against the edges kept so
    far (kept as sorted runs), so a round costs its own size."""
    if m > nu * nv:
        raise ValueError("more edges than cells")
    rng = np.random.default_rng(seed)
    cu = np.cumsum(_probs(nu, gamma_u, i0_u, m, nv))
    cv = np.cumsum(_probs(nv, gamma_v, i0_v, m, nu))
    cu /= cu[-1]
    cv /= cv[-1]
    parts, runs, have = [], [], 0
    for _ in range(1000):
        need = m - have
        if need <= 0:
            break
        k = int(need * 1.15) + 1024
        u = _draw(cu, rng, k)
        v = _draw(cv, rng, k)
        cand = u * nv + v
        new = cand[_first_new(runs, cand)[:need]]
        parts.append(new)
        runs.append(np.sort(new))
        have += len(new)
    if have < m:
        raise RuntimeError("could not draw enough distinct edges")
    keys = np.concatenate(parts) if parts else np.empty(0, dtype=np.int64)
    return (keys // nv).astype(np.int32), (keys % nv).astype(np.int32)


def complete_bipartite(a: int, b: int):
    """K_{a,b}: every U vertex adjacent to every V vertex."""
    eu = np.repeat(np.arange(a, dtype=np.int32), b)
    ev = np.tile(np.arange(b, dtype=np.int32), a)
    return eu, ev


def random_small(nu: int, nv: int, p: float, seed: int):
    """Tiny Bernoulli(p) bipartite graph (test fixture)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((nu, nv)) < p
    eu, ev = np.nonzero(mask)
    return eu.astype(np.int32), ev.astype(np.int32)


# --------------------------------------------------------------------------
# The named workloads
# --------------------------------------------------------------------------

ER_20K = "er-2000x500-20k"
CHUNG_LU_10M = "chung-lu-1Mx200k-10M"
CHUNG_LU_100M = "chung-lu-5Mx1M-100M"
# the 100M-edge graph's shape at a fifth of its size (profiling stand-in)
CHUNG_LU_20M = "chung-lu-2Mx400k-20M"

WORKLOADS = {
    ER_20K: dict(kind="er", nu=2000, nv=500, m=20000, seed=1, side=0),
    CHUNG_LU_10M: dict(kind="cl", nu=1_000_000, nv=200_000, m=10_000_000, gamma_u=2.5,
                       gamma_v=2.1, seed=2, dmax_v=50_000, side=0),
    CHUNG_LU_100M: dict(kind="cl", nu=5_000_000, nv=1_000_000, m=100_000_000, gamma_u=2.0,
                        gamma_v=2.0, seed=3, dmax_u=500_000, dmax_v=500_000, side=1),
    CHUNG_LU_20M: dict(kind="cl", nu=2_000_000, nv=400_000, m=20_000_000, gamma_u=2.0,
                       gamma_v=2.0, seed=33, dmax_u=100_000, dmax_v=100_000, side=1),
}


def _cache_dir():
    d = os.environ.get("RECEIPT_GRAPH_CACHE")
    if not d:
        d = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".graph_cache")
    os.makedirs(d, exist_ok=True)
    return d


def workload_graph(name: str, cache: bool = True):
    """Edge list of a named workload: ER_20K (Erdos-Renyi 2,000x500, 20k
    edges), CHUNG_LU_10M (Chung-Lu 1Mx200k, 10M edges, exponents 2.5/2.1, max
    V degree ~50k), CHUNG_LU_100M (Chung-Lu 5Mx1M, 100M edges, exponent 2.0 on
    both sides, hubs ~500k).

    Returns ``(eu, ev, nu, nv, side)``. Large graphs are cached as ``.npz``
    under ``$RECEIPT_GRAPH_CACHE`` (default ``.graph_cache`` beside the package)."""
    c = WORKLOADS[name]
    small = c["kind"] == "er"
    path = os.path.join(_cache_dir(), f"{name}.npz")
    if cache and not small and os.path.exists(path):
        z = np.load(path)
        return z["eu"], z["ev"], c["nu"], c["nv"], c["side"]
    if c["kind"] == "er":
        eu, ev = er(c["nu"], c["nv"], c["m"], c["seed"])
    else:
        i0u = 1.0
        if "dmax_u" in c:
            i0u = chung_lu_i0_for_max(c["nu"], c["gamma_u"], c["m"], c["dmax_u"])
        i0v = 1.0
        if "dmax_v" in c:
            i0v = chung_lu_i0_for_max(c["nv"], c["gamma_v"], c["m"], c["dmax_v"])
        eu, ev = chung_lu(c["nu"], c["nv"], c["m"], c["gamma_u"], c["gamma_v"],
                          c["seed"], i0u, i0v)
    if cache and not small:
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, eu=eu, ev=ev)
        os.replace(tmp, path)
    return eu, ev, c["nu"], c["nv"], c["side"]


@dataclass
class GraphSpec:
    """Size recipe of one graph of the batched or serving workload."""
    nu: int
    nv: int
    m: int
    gamma: float
    side: int
    seed: int


def batch_specs(n: int = 4096, seed: int = 4):
    """Batched workload: ``|U|`` log-uniform in [100, 20000], ``|V| = |U|//4``,
    ``m`` log-uniform in [1e3, 2e5] clamped to ``|U||V|/4``, exponent uniform
    in [2, 3] shared by both sides, ``i0 = 1``, U side decomposed."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(n):
        nu = int(round(math.exp(rng.uniform(math.log(100), math.log(20000)))))
        nv = max(1, nu // 4)
        m = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
        m = max(1, min(m, (nu * nv) // 4))
        gamma = float(rng.uniform(2.0, 3.0))
        out.append(GraphSpec(nu, nv, m, gamma, 0, int(rng.integers(1 << 62))))
    return out


def serve_specs(n: int = 10000, seed: int = 5):
    """Serving workload: ``m`` log-uniform in [1e4, 1e7], ratio ``r`` uniform in
    [1, 10], ``|U| = m/10``, ``|V| = |U|/r``, exponent uniform in [2, 3] on both
    sides, side chosen uniformly. Arrival times are drawn by the caller at a
    rate it chooses (``poisson_arrivals``)."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(n):
        m = int(round(math.exp(rng.uniform(math.log(1e4), math.log(1e7)))))
        r = float(rng.uniform(1.0, 10.0))
        nu = max(2, int(round(m / 10)))
        nv = max(2, int(round(nu / r)))
        m = max(1, min(m, (nu * nv) // 4))
        gamma = float(rng.uniform(2.0, 3.0))
        side = int(rng.integers(2))
        out.append(GraphSpec(nu, nv, m, gamma, side, int(rng.integers(1 << 62))))
    return out


def poisson_arrivals(n: int, rate: float, seed: int = 5):
    """Arrival times (seconds from t=0) of a Poisson stream of ``n`` requests."""
    rng = np.random.default_rng(seed + 1_000_003)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def graph_from_spec(s: GraphSpec):
    """Draw the Chung-Lu graph of one batch/serving spec."""
    return chung_lu(s.nu, s.nv, s.m, s.gamma, s.gamma, s.seed)
