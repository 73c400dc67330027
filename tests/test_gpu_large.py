"""Parity at the full workload sizes: the 100M-edge graph (Chung-Lu 5M x 1M,
exponent 2.0 on both sides, hubs of ~200k edges; V side decomposed, ~1.06e12
bottom-up wedges), the 4,096-graph batch and a prefix of the serving stream.

Drawing these graphs takes minutes on the host, so these tests run only when
RECEIPT_LARGE_TESTS=1. Butterfly counts of both sides are compared with the
oracle's digests (2-hop definition) and a seeded sample of single values;
tip numbers with the oracle's digest once `make_golden.py` has stored it,
and always with properties that hold at any size: 0 <= tip <= count, and
Theorem 1 (every vertex's tip number lies in its subset's range)."""
import hashlib
import json
import os

import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(
    os.environ.get("RECEIPT_LARGE_TESTS") != "1", reason="set RECEIPT_LARGE_TESTS=1")]

HERE = os.path.dirname(os.path.abspath(__file__))


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_08695_gb300 as R
    R.load()
    return R


@pytest.fixture(scope="module")
def chung_lu_100m():
    path = os.path.join(HERE, "golden", synth.CHUNG_LU_100M + ".json")
    if not os.path.exists(path):
        pytest.skip("oracle digests of the 100M-edge workload not generated")
    gold = json.load(open(path))
    eu, ev, nu, nv, side = synth.workload_graph(synth.CHUNG_LU_100M)
    assert synth.edges_sha256(eu, ev) == gold["edges_sha256"], "generator drew a different graph"
    return gold, eu, ev, nu, nv, side


def test_chung_lu_100m_counts_and_tips(R, chung_lu_100m):
    gold, eu, ev, nu, nv, side = chung_lu_100m
    g = R.Graph(eu, ev, nu, nv)
    cu, cv = g.count_butterflies()
    cu, cv = R.as_u64(cu), R.as_u64(cv)
    for k, v in gold["sample_u"].items():
        assert int(cu[int(k)]) == v
    for k, v in gold["sample_v"].items():
        assert int(cv[int(k)]) == v
    assert _sha(cu) == gold["count_u_sha256"]
    assert _sha(cv) == gold["count_v_sha256"]
    t, sub, bounds = g.tip_decompose(side, subsets=True)
    t = R.as_u64(t)
    cnt = cv if side == 1 else cu
    assert (t <= cnt).all()
    sub = sub.cpu().numpy()
    assert (bounds[sub] <= t).all() and (t < bounds[sub + 1]).all()
    if "tips_sha256" in gold:
        for k, v in gold["sample_tips"].items():
            assert int(t[int(k)]) == v, f"vertex {k}"
        assert _sha(t) == gold["tips_sha256"]


def _draw_all(specs):
    """Draws spec'd graphs in spawned host processes (no fork after CUDA)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        return pool.map(synth.graph_from_spec, specs, chunksize=8)


def test_batch_of_4096_graphs(R):
    """The seed-4 batch of 4,096 graphs (94.7M edges) in one
    receipt_decompose_batch call, as the batch benchmark launches it: every
    graph's tips equal its own decomposition, a seeded sample the oracle's."""
    specs = synth.batch_specs(4096, seed=4)
    graphs = _draw_all(specs)
    built = [R.Graph(eu, ev, s.nu, s.nv) for (eu, ev), s in zip(graphs, specs)]
    outs = R.receipt_decompose_batch(built, [0] * len(built))
    for i, g in enumerate(built):
        assert np.array_equal(R.as_u64(outs[i]), R.as_u64(g.tip_decompose(0))), f"graph {i}"
    rng = np.random.default_rng(404)
    for i in sorted(rng.choice(len(built), 32, replace=False)):
        (eu, ev), s = graphs[i], specs[i]
        assert np.array_equal(R.as_u64(outs[i]), oracle.bup(eu, ev, s.nu, s.nv, 0)[0]), \
            f"graph {i}"


def test_serving_stream_prefix(R):
    """The first 200 requests of the seed-5 serving stream submitted at once:
    every tenth result equals the request decomposed alone, and the requests
    of at most 200k edges among the first 100 equal the oracle's."""
    specs = synth.serve_specs(200, seed=5)
    graphs = _draw_all(specs)
    reqs = [(eu, ev, s.nu, s.nv, s.side) for (eu, ev), s in zip(graphs, specs)]
    sv = R.Server(max_inflight=4)
    ids = [sv.submit(*r)[0] for r in reqs]
    outs = [sv.wait(i)[0] for i in ids]
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for i in range(0, len(reqs), 10):
        assert np.array_equal(outs[i], R.receipt_tip_decompose_host(*reqs[i])), f"request {i}"
    for i in range(100):
        if len(reqs[i][0]) <= 200000:
            assert np.array_equal(outs[i], oracle.bup(*reqs[i])[0]), f"request {i}"
