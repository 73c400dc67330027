"""Parity on the 100M-edge workload (Chung-Lu 5M x 1M, exponent 2.0 on both
sides, hubs of ~200k edges; V side decomposed, ~1.06e12 bottom-up wedges).

Drawing the graph takes minutes on one core, so these tests run only when
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
