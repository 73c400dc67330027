"""Parity of the CUDA path (through the C ABI) with the CPU oracle: butterfly
counts and tip numbers must match bit for bit, on seeded synthetic graphs
that exercise every aggregation tier (warp table, shared-memory hybrid,
global dense counters), both sides, empty and degenerate inputs, and the
theorems the method rests on (Theorem 2: any ranges give the same tip
numbers; Theorem 1: every vertex's tip number lies in its subset's range)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_08695_gb300 as R
    R.load()
    return R


def _gpu_counts(R, eu, ev, nu, nv):
    g = R.Graph(eu, ev, nu, nv)
    cu, cv = g.count_butterflies()
    return R.as_u64(cu), R.as_u64(cv)


def _gpu_tips(R, eu, ev, nu, nv, side, **kw):
    g = R.Graph(eu, ev, nu, nv)
    t = g.tip_decompose(side, **kw)
    return R.as_u64(t), g


def _check_graph(R, eu, ev, nu, nv, sides=(0, 1)):
    cu, cv = oracle.count_2hop(eu, ev, nu, nv)
    gu, gv = _gpu_counts(R, eu, ev, nu, nv)
    assert np.array_equal(gu, cu), "U counts differ"
    assert np.array_equal(gv, cv), "V counts differ"
    for side in sides:
        want, _ = oracle.bup(eu, ev, nu, nv, side)
        got, g = _gpu_tips(R, eu, ev, nu, nv, side)
        bad = np.nonzero(got != want)[0]
        assert len(bad) == 0, f"side {side}: {len(bad)} tips differ, e.g. {bad[:5]} " \
                              f"got {got[bad[:5]]} want {want[bad[:5]]}"
        # next activeSets from the support atomics' returned values, sliced
        # tier at one CTA per SM, no vertex cap on the ranges
        got = R.as_u64(g.tip_decompose(side, scan_frontier=-1, slice_ctas=1, range_max_n=-1))
        assert np.array_equal(got, want), f"side {side}: crossings / slice_ctas=1 / no cap"
        # a tight vertex cap on the ranges
        got = R.as_u64(g.tip_decompose(side, range_max_n=max(1, (nu, nv)[side] // 500)))
        assert np.array_equal(got, want), f"side {side}: range_max_n"


def test_tiny_random_graphs(R):
    rng = np.random.default_rng(101)
    for _ in range(40):
        nu, nv = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        eu, ev = synth.random_small(nu, nv, float(rng.uniform(0.1, 0.9)), int(rng.integers(1 << 30)))
        _check_graph(R, eu, ev, nu, nv)


def test_er_20k_golden(R):
    eu, ev, nu, nv, side = synth.workload_graph(synth.ER_20K)
    gold = json.load(open(os.path.join(HERE, "golden", synth.ER_20K + ".json")))
    assert synth.edges_sha256(eu, ev) == gold["edges_sha256"]
    _check_graph(R, eu, ev, nu, nv)


@pytest.mark.parametrize("seed,nu,nv,m,gu,gv", [
    (11, 30000, 6000, 200000, 2.5, 2.1),
    (12, 5000, 20000, 150000, 2.1, 2.6),
    (13, 60000, 2000, 300000, 2.3, 2.0),
])
def test_chung_lu_medium(R, seed, nu, nv, m, gu, gv):
    eu, ev = synth.chung_lu(nu, nv, m, gu, gv, seed)
    _check_graph(R, eu, ev, nu, nv)


def test_repeat_table_overflow_path(R):
    # every U vertex has ~10 neighbours among 200 V vertices of degree ~2000:
    # thousands of repeated end points per anchor, beyond the shared table
    eu, ev = synth.er(40000, 200, 400000, seed=21)
    _check_graph(R, eu, ev, 40000, 200, sides=(0,))


def test_sliced_tier_over_several_key_slices(R):
    # 150k U vertices (three 64K-key slices); a low slice threshold sends every
    # anchor with more than 2,000 wedges through the sliced tier, and a tiny
    # threshold also exercises its repeat-table fallback
    eu, ev = synth.chung_lu(150000, 3000, 450000, 2.4, 2.3, seed=41)
    want, _ = oracle.bup(eu, ev, 150000, 3000, 0)
    g = R.Graph(eu, ev, 150000, 3000)
    for smw in (2000, 300):
        t = R.as_u64(g.tip_decompose(0, slice_min_w=smw, timing=True))
        assert np.array_equal(t, want), f"slice_min_w={smw}"
        st = g.stats()
        assert st["peel_anchors"][3] > 0
    # the tier's three shapes (1, 2 and 4 CTAs per SM over 2, 4 and 7 key
    # slices here), with the next activeSet from crossings or from scans
    for ctas in (1, 2, 4):
        for scan in (-1, 1):
            t = R.as_u64(g.tip_decompose(0, slice_min_w=2000, slice_ctas=ctas,
                                         scan_frontier=scan, timing=True))
            assert np.array_equal(t, want), f"slice_ctas={ctas} scan={scan}"
            assert g.stats()["peel_anchors"][3] > 0
    t = R.as_u64(g.tip_decompose(0, warp_max_w=32))
    assert np.array_equal(t, want)
    # one subset of 150k ranks: the fine-grained step aggregates rank slices
    t = R.as_u64(g.tip_decompose(0, P=1))
    assert np.array_equal(t, want)


def test_hub_with_degree_above_16_bits(R):
    rng = np.random.default_rng(22)
    nu, nv = 80000, 50
    eu = [np.arange(70000, dtype=np.int32)]
    ev = [np.zeros(70000, np.int32)]
    for v in range(1, nv):
        us = rng.choice(nu, 1200, replace=False).astype(np.int32)
        eu.append(us)
        ev.append(np.full(len(us), v, np.int32))
    eu, ev = np.concatenate(eu), np.concatenate(ev)
    _check_graph(R, eu, ev, nu, nv, sides=(1,))


def test_complete_bipartite_and_degenerate(R):
    for a, b in [(1, 1), (2, 2), (9, 7), (64, 33), (300, 5)]:
        eu, ev = synth.complete_bipartite(a, b)
        t, _ = _gpu_tips(R, eu, ev, a, b, 0)
        assert (t == (a - 1) * (b * (b - 1) // 2)).all()
        t, _ = _gpu_tips(R, eu, ev, a, b, 1)
        assert (t == (b - 1) * (a * (a - 1) // 2)).all()
    # empty graph, isolated vertices, single edge, empty side
    e = np.zeros(0, np.int32)
    t, _ = _gpu_tips(R, e, e, 5, 3, 0)
    assert (t == 0).all() and len(t) == 5
    t, _ = _gpu_tips(R, e, e, 0, 3, 0)
    assert len(t) == 0
    t, _ = _gpu_tips(R, np.array([2], np.int32), np.array([1], np.int32), 4, 3, 1)
    assert (t == 0).all()
    # a star and a hub adjacent to everything
    eu = np.zeros(100, np.int32)
    ev = np.arange(100, dtype=np.int32)
    _check_graph(R, eu, ev, 1, 100)
    eu, ev = synth.er(300, 40, 2000, seed=5)
    eu = np.concatenate([eu, np.full(300, 0, np.int32)])
    ev = np.concatenate([ev, np.arange(300, dtype=np.int32) % 40])
    eu, ev = np.concatenate([eu, np.arange(300, dtype=np.int32)]), \
        np.concatenate([ev, np.full(300, 39, np.int32)])
    _check_graph(R, eu, ev, 300, 40)


def test_equal_degrees_regular(R):
    # 2-regular cycle-like bipartite graph and a 3-regular circulant
    n = 500
    u = np.arange(n, dtype=np.int32)
    for k in (2, 3):
        eu = np.concatenate([u] * k)
        ev = np.concatenate([(u + j) % n for j in range(k)]).astype(np.int32)
        _check_graph(R, eu, ev, n, n)


def test_duplicates_and_errors(R):
    eu = np.array([0, 0, 1, 1, 0, 1], np.int32)
    ev = np.array([0, 1, 0, 1, 0, 1], np.int32)
    t, g = _gpu_tips(R, eu, ev, 3, 2, 0)
    assert t.tolist() == [1, 1, 0] and g.m == 4
    with pytest.raises(R.ReceiptError) as ei:
        R.Graph(eu, ev, 3, 2, dedup=False)
    assert ei.value.status == 1
    with pytest.raises(R.ReceiptError) as ei:
        R.Graph(np.array([3], np.int32), np.array([0], np.int32), 3, 2)
    assert ei.value.status == 1
    g = R.Graph(eu, ev, 3, 2)
    with pytest.raises(R.ReceiptError):
        g.tip_decompose(side=2)


def test_any_P_and_injected_ranges_give_same_tips(R):
    eu, ev = synth.chung_lu(20000, 4000, 120000, 2.4, 2.2, seed=31)
    want, _ = oracle.bup(eu, ev, 20000, 4000, 0)
    g = R.Graph(eu, ev, 20000, 4000)
    for P in (1, 2, 7, 150, 600):
        t, sub, bounds = g.tip_decompose(0, P=P, subsets=True)
        t = R.as_u64(t)
        assert np.array_equal(t, want), f"P={P}"
        sub = sub.cpu().numpy()
        # Theorem 1: theta(i) <= tip < theta(i+1) for every vertex of U_i
        lo = bounds[sub]
        hi = bounds[sub + 1]
        assert (lo <= t).all() and (t < hi).all(), f"P={P}"
    t = R.as_u64(g.tip_decompose(0, dgm=False))  # without dynamic graph maintenance
    assert np.array_equal(t, want)
    t = R.as_u64(g.tip_decompose(0, round_graphs=True))  # rounds as CUDA graph launches
    assert np.array_equal(t, want)
    assert g.stats()["rounds_cd"] >= 1
    rng = np.random.default_rng(3)
    top = int(want.max()) + 2
    for trial in range(4):
        k = int(rng.integers(1, 12))
        b = np.unique(rng.integers(1, top, size=k)).astype(np.uint64)
        t, sub, bounds = g.tip_decompose(0, P=len(b), bounds=b, subsets=True)
        assert np.array_equal(R.as_u64(t), want), f"bounds {b}"


def _round_records(tr):
    return [(r["range"], r["frontier"], r["hi"], r["recount"], tuple(r["anchors"]),
             tuple(r["wedges"])) for r in tr]


def test_round_launch_modes_give_same_rounds(R):
    # device-driven rounds (default: while-node graph launches of up to 64
    # rounds), one graph launch per round, separate launches per round: same
    # tip numbers and the same per-round records
    eu, ev = synth.chung_lu(20000, 4000, 120000, 2.4, 2.2, seed=31)
    g = R.Graph(eu, ev, 20000, 4000)
    for side in (0, 1):
        want, _ = oracle.bup(eu, ev, 20000, 4000, side)
        for P, huc in ((1, 0), (7, 0), (150, 0), (40, 1)):
            recs = []
            for mode in (0, True, -1):
                t = R.as_u64(g.tip_decompose(side, P=P, huc=huc, round_graphs=mode))
                assert np.array_equal(t, want), f"side {side} P={P} huc={huc} mode {mode}"
                recs.append(_round_records(g.trace()))
                assert g.stats()["rounds_cd"] == len(recs[-1])
            assert recs[0] == recs[1] == recs[2], f"side {side} P={P} huc={huc}"
    # a ladder: u_i shares one butterfly with u_{i-1} and one with u_{i+1},
    # so below the bound 2 the peel cascades in from both ends, two vertices
    # a round: one range of ~k/2 rounds, several launches of the while-node
    k = 400
    i = np.arange(k, dtype=np.int32)
    eu = np.repeat(i, 4)
    ev = np.stack([i, i + 1, k + 1 + i, k + 2 + i], axis=1).reshape(-1).astype(np.int32)
    g = R.Graph(eu, ev, k, 2 * (k + 1))
    want, _ = oracle.bup(eu, ev, k, 2 * (k + 1), 0)
    recs = []
    for mode in (0, True, -1):
        t = R.as_u64(g.tip_decompose(0, P=1, bounds=np.array([2], np.uint64), round_graphs=mode))
        assert np.array_equal(t, want), f"ladder mode {mode}"
        recs.append(_round_records(g.trace()))
    assert recs[0] == recs[1] == recs[2]
    assert len(recs[0]) >= 3 * 64


def test_heavy_subset_path_gives_same_tips(R):
    """Subsets peeled by all CTAs level by level (forced for every subset,
    or never) give the one-CTA result; the per-subset records add up."""
    eu, ev = synth.chung_lu(20000, 4000, 120000, 2.4, 2.2, seed=33)
    want, _ = oracle.bup(eu, ev, 20000, 4000, 0)
    g = R.Graph(eu, ev, 20000, 4000)
    for P in (1, 5, 150):
        for hw in (1, -1, 0):
            t = R.as_u64(g.tip_decompose(0, P=P, fd_heavy_w=hw))
            assert np.array_equal(t, want), f"P={P} fd_heavy_w={hw}"
            st, subs = g.stats(), g.subsets()
            assert len(subs) == st["p_eff"]
            assert sum(s["n"] for s in subs) == 20000
            heavy = [s for s in subs if s["heavy"]]
            assert len(heavy) == st["fd_heavy_subsets"]
            if hw == 1:
                assert len(heavy) == sum(1 for s in subs if s["n"] > 0 and s["wedges_est"] >= 1)
                if P == 1:  # levels with few big walks spread them over the CTAs
                    assert 0 < st["fd_split_levels"] <= st["levels_fd_heavy"]
            if hw == -1:
                assert st["fd_split_levels"] == 0
            if hw == -1:
                assert not heavy
            assert sum(s["levels"] for s in subs) == st["levels_fd"]
            assert sum(s["levels"] for s in heavy) == st["levels_fd_heavy"]
    # V side of a graph with a hub of degree >= 2^16 (32-bit counters) and a
    # side of 150k ranks in one subset (several rank slices), heavy path forced
    rng = np.random.default_rng(22)
    nu, nv = 80000, 50
    eu = [np.arange(70000, dtype=np.int32)]
    ev = [np.zeros(70000, np.int32)]
    for v in range(1, nv):
        us = rng.choice(nu, 1200, replace=False).astype(np.int32)
        eu.append(us)
        ev.append(np.full(len(us), v, np.int32))
    eu, ev = np.concatenate(eu), np.concatenate(ev)
    want, _ = oracle.bup(eu, ev, nu, nv, 1)
    got, _ = _gpu_tips(R, eu, ev, nu, nv, 1, fd_heavy_w=1)
    assert np.array_equal(got, want)
    eu, ev = synth.chung_lu(150000, 3000, 600000, 2.3, 2.1, seed=34)
    want, _ = oracle.bup(eu, ev, 150000, 3000, 0)
    got, _ = _gpu_tips(R, eu, ev, 150000, 3000, 0, P=1, fd_heavy_w=1)
    assert np.array_equal(got, want)


def test_recount_rounds_give_same_tips(R):
    """Hybrid update computation (Sec. 4.1): ranges whose first round
    recounts the remaining subgraph instead of peeling (forced for every
    range, or chosen by the cost rule with a tiny factor) give the oracle's
    tips on both sides, for any P, with dynamic graph maintenance on and off,
    with rounds as graph launches and injected ranges; C_rcnt equals the sum
    over edges of min(d_u, d_v)."""
    nu, nv = 20000, 4000
    eu, ev = synth.chung_lu(nu, nv, 120000, 2.4, 2.2, seed=35)
    du, dv = np.bincount(eu, minlength=nu), np.bincount(ev, minlength=nv)
    crcnt = int(np.minimum(du[eu], dv[ev]).sum())
    g = R.Graph(eu, ev, nu, nv)
    for side in (0, 1):
        want, _ = oracle.bup(eu, ev, nu, nv, side)
        for P in (1, 3, 40, 150):
            for dgm in (True, False):
                t = R.as_u64(g.tip_decompose(side, P=P, huc=1, dgm=dgm, timing=True))
                assert np.array_equal(t, want), f"side {side} P={P} dgm={dgm}"
                st, tr = g.stats(), g.trace()
                ranges = sorted({r["range"] for r in tr})
                assert st["huc_recounts"] == len(ranges) >= 1
                firsts = {}
                for r in tr:
                    firsts.setdefault(r["range"], r)
                assert all(r["recount"] == (firsts[r["range"]] is r) for r in tr)
                assert all(sum(r["wedges"]) == 0 for r in tr if r["recount"])
                if P > 1:  # with one range the first activeSet takes every vertex
                    assert st["wedges_recount"] > 0 and st["ms_recount"] > 0
        t = R.as_u64(g.tip_decompose(side, huc=1, round_graphs=True))
        assert np.array_equal(t, want), f"side {side} graph rounds"
        b = np.array([3, 50, 400, 5000], np.uint64)
        t = R.as_u64(g.tip_decompose(side, P=len(b), bounds=b, huc=1))
        assert np.array_equal(t, want), f"side {side} injected ranges"
        t = R.as_u64(g.tip_decompose(side, P=20, huc=0, huc_factor_1024=1))
        assert np.array_equal(t, want), f"side {side} rule with factor 1/1024"
        st = g.stats()
        assert st["cost_recount"] == crcnt and st["huc_recounts"] >= 1
        g.tip_decompose(side, huc=-1)
        st = g.stats()
        assert st["huc_recounts"] == 0 and st["cost_recount"] == 0
    # a hub of degree >= 2^16 on the other side: the recount goes through the
    # counting kernels' global-counter tier
    rng = np.random.default_rng(36)
    nu, nv = 80000, 40
    eu = [np.arange(70000, dtype=np.int32)]
    ev = [np.zeros(70000, np.int32)]
    for v in range(1, nv):
        us = rng.choice(nu, 900, replace=False).astype(np.int32)
        eu.append(us)
        ev.append(np.full(len(us), v, np.int32))
    eu, ev = np.concatenate(eu), np.concatenate(ev)
    want, _ = oracle.bup(eu, ev, nu, nv, 1)
    got, _ = _gpu_tips(R, eu, ev, nu, nv, 1, P=4, huc=1)
    assert np.array_equal(got, want), "hub graph"
    # a batch of graphs packed into one union
    specs = synth.batch_specs(16, seed=37)
    graphs, wants = [], []
    for s in specs:
        beu, bev = synth.graph_from_spec(s)
        graphs.append(R.Graph(beu, bev, s.nu, s.nv))
        wants.append(oracle.bup(beu, bev, s.nu, s.nv, 0)[0])
    outs = R.receipt_decompose_batch(graphs, [0] * len(graphs), huc=1)
    for i, (o, w) in enumerate(zip(outs, wants)):
        assert np.array_equal(R.as_u64(o), w), f"batch graph {i}"
    assert graphs[0].stats()["huc_recounts"] >= 1


def test_fd_recount_levels_give_same_tips(R):
    """Hybrid update computation inside the fine-grained step (Sec. 4.1):
    heavy tasks (all tasks forced heavy) whose levels recount the task's
    alive members instead of applying updates -- at every level, or by the
    cost rule with a tiny factor -- give the oracle's tips on both sides,
    for one subset and for several, and in a batch."""
    nu, nv = 3000, 800
    eu, ev = synth.chung_lu(nu, nv, 20000, 2.3, 2.2, seed=36)
    g = R.Graph(eu, ev, nu, nv)
    for side in (0, 1):
        want, _ = oracle.bup(eu, ev, nu, nv, side)
        for P in (1, 3, 12):
            t = R.as_u64(g.tip_decompose(side, P=P, fd_heavy_w=1, fd_huc=1))
            assert np.array_equal(t, want), f"side {side} P={P} forced"
            st = g.stats()
            assert st["fd_heavy_subsets"] > 0 and st["fd_recounts"] > 0
            t = R.as_u64(g.tip_decompose(side, P=P, fd_heavy_w=1, fd_huc=0, huc_factor_1024=1))
            assert np.array_equal(t, want), f"side {side} P={P} rule"
            assert g.stats()["fd_recounts"] > 0
    # never: no recount
    t = R.as_u64(g.tip_decompose(0, P=3, fd_heavy_w=1, fd_huc=-1))
    assert g.stats()["fd_recounts"] == 0
    # a batch: tasks are packed graphs' parts of a subset
    parts = [synth.chung_lu(400 + 50 * k, 120, 2500, 2.3, 2.2, seed=60 + k) for k in range(5)]
    built = [R.Graph(a, b, 400 + 50 * k, 120) for k, (a, b) in enumerate(parts)]
    outs = R.receipt_decompose_batch(built, [0] * 5, P=4, fd_heavy_w=1, fd_huc=1)
    for k, ((a, b), o) in enumerate(zip(parts, outs)):
        assert np.array_equal(R.as_u64(o), oracle.bup(a, b, 400 + 50 * k, 120, 0)[0]), f"graph {k}"


def test_batch_equals_alone(R):
    specs = synth.batch_specs(24, seed=4)
    graphs, sides, wants = [], [], []
    for i, s in enumerate(specs):
        eu, ev = synth.graph_from_spec(s)
        side = i % 2
        graphs.append(R.Graph(eu, ev, s.nu, s.nv))
        sides.append(side)
        wants.append(oracle.bup(eu, ev, s.nu, s.nv, side)[0])
    outs = R.receipt_decompose_batch(graphs, sides)
    for i, (o, w) in enumerate(zip(outs, wants)):
        assert np.array_equal(R.as_u64(o), w), f"graph {i}"
    outs = R.receipt_decompose_batch(graphs, sides, round_graphs=True)
    for i, (o, w) in enumerate(zip(outs, wants)):
        assert np.array_equal(R.as_u64(o), w), f"graph {i} (graph rounds)"
        alone = R.as_u64(graphs[i].tip_decompose(sides[i]))
        assert np.array_equal(alone, w)


def test_large_batch_of_small_graphs(R):
    """Hundreds of small graphs in one union: rounds with more dense-window
    anchors than CTAs (several anchors per pass) and FD tasks per graph part;
    every graph's tips equal its own decomposition, a sample the oracle's."""
    rng = np.random.default_rng(44)
    graphs, wants, edges = [], [], []
    for i in range(600):
        nu = int(rng.integers(60, 900))
        nv = int(rng.integers(20, 300))
        m = int(min(rng.integers(200, 6000), nu * nv // 3))
        eu, ev = synth.chung_lu(nu, nv, m, 2.3, 2.1, seed=int(rng.integers(1 << 30)))
        graphs.append(R.Graph(eu, ev, nu, nv))
        edges.append((eu, ev, nu, nv))
    outs = R.receipt_decompose_batch(graphs, [0] * len(graphs))
    st = graphs[0].stats()
    assert st["fd_tasks"] > st["p_eff"]  # subsets were split by graph
    for i, g in enumerate(graphs):
        alone = R.as_u64(g.tip_decompose(0))
        assert np.array_equal(R.as_u64(outs[i]), alone), f"graph {i}"
    for i in range(0, len(graphs), 60):
        eu, ev, nu, nv = edges[i]
        assert np.array_equal(R.as_u64(outs[i]), oracle.bup(eu, ev, nu, nv, 0)[0]), f"graph {i}"


def test_host_buffer_entry(R):
    eu, ev, nu, nv, side = synth.workload_graph(synth.ER_20K)
    got = R.receipt_tip_decompose_host(eu, ev, nu, nv, 0)
    want, _ = oracle.bup(eu, ev, nu, nv, 0)
    assert np.array_equal(got, want)


def test_stats_are_reported(R):
    eu, ev, nu, nv, side = synth.workload_graph(synth.ER_20K)
    g = R.Graph(eu, ev, nu, nv)
    g.tip_decompose(0, timing=True)
    st = g.stats()
    assert st["p_eff"] >= 1 and st["rounds_cd"] >= 1 and st["wedges_count"] > 0
    assert st["ms_total"] > 0


def test_chung_lu_10m_golden(R):
    path = os.path.join(HERE, "golden", synth.CHUNG_LU_10M + ".json")
    if not os.path.exists(path):
        pytest.skip("golden digests of the 10M-edge workload not generated")
    gold = json.load(open(path))
    eu, ev, nu, nv, side = synth.workload_graph(synth.CHUNG_LU_10M)
    assert synth.edges_sha256(eu, ev) == gold["edges_sha256"], "generator drew a different graph"
    import hashlib
    g = R.Graph(eu, ev, nu, nv)
    cu, cv = g.count_butterflies()
    cu, cv = R.as_u64(cu), R.as_u64(cv)
    for k, v in gold["sample_u"].items():
        assert int(cu[int(k)]) == v
    for k, v in gold["sample_v"].items():
        assert int(cv[int(k)]) == v
    assert hashlib.sha256(cu.astype("<u8").tobytes()).hexdigest() == gold["count_u_sha256"]
    assert hashlib.sha256(cv.astype("<u8").tobytes()).hexdigest() == gold["count_v_sha256"]
    t = R.as_u64(g.tip_decompose(side))
    for k, v in gold["sample_tips"].items():
        assert int(t[int(k)]) == v, f"vertex {k}"
    assert hashlib.sha256(t.astype("<u8").tobytes()).hexdigest() == gold["tips_sha256"]
