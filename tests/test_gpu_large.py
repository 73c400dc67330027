"""Parity at the full workload sizes, run by default under `pytest -m gpu`.

* the 100M-edge graph (Chung-Lu 5M x 1M, exponent 2.0 on both sides, hubs
  of ~200k edges; V side decomposed, ~1.06e12 bottom-up wedges): butterfly
  counts of both sides and tip numbers against the oracle's stored digests
  (`tests/golden/chung-lu-5Mx1M-100M.json`, written by `make_golden.py`
  from the oracle alone) and seeded single values, plus 0 <= tip <= count
  and Theorem 1 (every tip number lies in its subset's range);
* the 4,096-graph batch (seed 4, 94.7M edges) in one
  receipt_decompose_batch call: every graph's tip numbers against the
  oracle's sequential peel of that graph (Algorithm 2);
* the first 200 requests of the seed-5 serving stream, all submitted at
  once: every result equals the request decomposed alone, and the oracle's
  for every request whose bottom-up wedge count is at most 1e9 (156 of the
  200).

Host-side drawing and the oracle runs go through spawned worker processes
(`large_inputs.py`)."""
import hashlib
import json
import os

import numpy as np
import pytest

import synth
from tests import large_inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SERVE_PREFIX = 200
SERVE_ORACLE_WEDGES = 10 ** 9


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
    for k, v in gold["sample_tips"].items():
        assert int(t[int(k)]) == v, f"vertex {k}"
    assert _sha(t) == gold["tips_sha256"]


def test_batch_of_4096_graphs(R):
    """The seed-4 batch as the batch benchmark launches it (one
    receipt_decompose_batch call, and once more with every coarse-grained
    round as a CUDA graph launch): every graph's tips equal the oracle's."""
    specs = synth.batch_specs(4096, seed=4)
    drawn = large_inputs.draw_all(specs, wedge_bound=float("inf"), chunksize=8)
    built = [R.Graph(eu, ev, s.nu, s.nv) for (eu, ev, _, _), s in zip(drawn, specs)]
    outs = R.receipt_decompose_batch(built, [0] * len(built))
    bad = [i for i, (o, d) in enumerate(zip(outs, drawn)) if not np.array_equal(R.as_u64(o), d[2])]
    assert not bad, f"{len(bad)} graphs differ from the oracle, first {bad[:8]}"
    again = R.receipt_decompose_batch(built, [0] * len(built), round_graphs=True)
    import torch
    assert all(torch.equal(a, b) for a, b in zip(outs, again))


def test_serving_stream_prefix(R):
    """The first 200 requests of the seed-5 serving stream, submitted at
    once (continuous batching packs and overlaps them)."""
    specs = synth.serve_specs(SERVE_PREFIX, seed=5)
    drawn = large_inputs.draw_all(specs, wedge_bound=SERVE_ORACLE_WEDGES)
    reqs = [(eu, ev, s.nu, s.nv, s.side) for (eu, ev, _, _), s in zip(drawn, specs)]
    sv = R.Server(max_inflight=4)
    ids = [sv.submit(*r)[0] for r in reqs]
    outs = [sv.wait(i)[0] for i in ids]
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for i, r in enumerate(reqs):
        assert np.array_equal(outs[i], R.receipt_tip_decompose_host(*r)), f"request {i}"
    checked = 0
    for i, d in enumerate(drawn):
        if d[2] is not None:
            assert np.array_equal(outs[i], d[2]), f"request {i} differs from the oracle"
            checked += 1
    assert checked >= SERVE_PREFIX * 3 // 4
