"""Serving engine (continuous batching): every request's tip numbers are the
same in the mix as alone (and as the oracle's, on a sample); small waiting
requests are packed together; several units overlap on the device; a
memory budget smaller than one request serialises admission."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_08695_gb300 as R
    R.load()
    return R


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if i % 7 == 3:  # a few larger requests among many small ones
            nu, nv, m = 20000, 4000, 150000
        else:
            nu = int(rng.integers(200, 3000))
            nv = int(rng.integers(50, 800))
            m = int(min(rng.integers(500, 20000), nu * nv // 4))
        gamma = float(rng.uniform(2.0, 3.0))
        eu, ev = synth.chung_lu(nu, nv, m, gamma, gamma, int(rng.integers(1 << 30)))
        out.append((eu, ev, nu, nv, int(rng.integers(2))))
    return out


def _alone(R, eu, ev, nu, nv, side):
    g = R.Graph(eu, ev, nu, nv)
    return R.as_u64(g.tip_decompose(side))


def test_mix_equals_alone_and_oracle(R):
    reqs = _requests(28, seed=5)
    sv = R.Server(max_inflight=4, batch_max_edges=25000, batch_max_graphs=16)
    ids = [sv.submit(*r)[0] for r in reqs]  # a flood: everything waits together
    got = [sv.wait(i)[0] for i in ids]
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["batches"] >= 1 and st["packed_requests"] >= 2
    assert st["peak_inflight"] >= 2
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for k, ((eu, ev, nu, nv, side), t) in enumerate(zip(reqs, got)):
        assert np.array_equal(t, _alone(R, eu, ev, nu, nv, side)), f"request {k}"
    for k in range(0, len(reqs), 5):
        eu, ev, nu, nv, side = reqs[k]
        assert np.array_equal(got[k], oracle.bup(eu, ev, nu, nv, side)[0]), f"request {k}"


def test_staggered_arrivals(R):
    reqs = _requests(12, seed=6)
    sv = R.Server(max_inflight=3)
    ids = []
    for r in reqs:
        ids.append(sv.submit(*r)[0])
        time.sleep(0.002)
    got = [sv.wait(i)[0] for i in ids]
    sv.close()
    for (eu, ev, nu, nv, side), t in zip(reqs, got):
        assert np.array_equal(t, _alone(R, eu, ev, nu, nv, side))


def test_memory_budget_serialises_admission(R):
    reqs = _requests(6, seed=7)
    sv = R.Server(max_inflight=4, mem_budget_bytes=1 << 20, batch_max_edges=0)
    ids = [sv.submit(*r)[0] for r in reqs]
    got = [sv.wait(i)[0] for i in ids]
    st = sv.stats()
    sv.close()
    assert st["peak_inflight"] == 1 and st["batches"] == 0
    for (eu, ev, nu, nv, side), t in zip(reqs, got):
        assert np.array_equal(t, _alone(R, eu, ev, nu, nv, side))


def test_bad_request_is_rejected(R):
    sv = R.Server(max_inflight=1)
    eu = np.array([5], np.int32)
    ev = np.array([0], np.int32)
    rid, _ = sv.submit(eu, ev, 3, 2, 0)  # id out of range: fails on the device path
    with pytest.raises(R.ReceiptError):
        sv.wait(rid)
    st = sv.stats()
    sv.close()
    assert st["failed"] == 1
