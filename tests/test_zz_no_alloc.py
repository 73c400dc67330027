"""Allocation-free butterfly counting (receipt_count_butterflies_noalloc).

For callers that may not allocate device memory while running, e.g. a
serving loop whose memory was reserved at start-up. The test calls the
entry point through the C ABI on three different graphs in a row (the
third with two hubs of degree 65,535, so the global-counter tier runs) and
on the first graph again, and compares each result with the allocating
entry point bit for bit (counts are exact integers); it also checks the size limits are enforced and that the
calls leave the device's free memory unchanged. This file is collected last.
"""
import numpy as np
import pytest

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


def _two_hubs():
    """65,536 x 2,000 graph in which V vertices 0 and 1 each have 65,535
    neighbours, plus 200,000 random edges. The hub that comes second in the
    degree order is a start point with degree >= 65,535, so its counts go
    through the global-counter slots carved out of the static array."""
    nu, nv = 65536, 2000
    hu = np.concatenate([np.arange(0, 65535), np.arange(1, 65536)]).astype(np.int32)
    hv = np.concatenate([np.zeros(65535), np.ones(65535)]).astype(np.int32)
    ru, rv = synth.er(nu, nv, 200000, seed=79)
    return (np.concatenate([hu, ru]), np.concatenate([hv, rv])), nu, nv


def _graphs():
    yield synth.chung_lu(40000, 9000, 300000, 2.3, 2.1, seed=77), 40000, 9000
    yield synth.er(6000, 1500, 120000, seed=78), 6000, 1500
    yield _two_hubs()


def test_noalloc_matches_allocating_entry_point_twice(R):
    import torch
    built = [(R.Graph(eu, ev, nu, nv), nu, nv) for (eu, ev), nu, nv in _graphs()]
    hubs = sorted(np.bincount(_two_hubs()[0][1], minlength=2000))[-2:]
    assert hubs[0] >= 65535 and built[2][0].max_degree[1] >= 65535
    refs = [g.count_butterflies() for g, _, _ in built]
    # outputs are the caller's: allocate them before watching free memory
    outs = [(torch.full((nu,), -1, dtype=torch.int64, device="cuda"),
             torch.full((nv,), -1, dtype=torch.int64, device="cuda")) for _, nu, nv in built]
    again = torch.full((built[0][1],), -1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for (g, nu, nv), (cu, cv) in zip(built, outs):
        R.receipt_count_butterflies_noalloc(g.handle, cu, cv)
    # the first graph again, after the other one used the shared scratch
    R.receipt_count_butterflies_noalloc(built[0][0].handle, again, None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free_before
    for (cu, cv), (ru, rv) in zip(outs, refs):
        assert torch.equal(cu, ru) and torch.equal(cv, rv)
    assert torch.equal(again, refs[0][0])


def test_noalloc_rejects_graphs_beyond_its_limits(R):
    eu = np.arange(70000, dtype=np.int32)
    ev = np.zeros(70000, dtype=np.int32)
    g = R.Graph(eu, ev, 70000, 1)
    import torch
    cu = torch.empty(70000, dtype=torch.int64, device="cuda")
    with pytest.raises(R.ReceiptError) as ei:
        R.receipt_count_butterflies_noalloc(g.handle, cu, None)
    assert ei.value.status == 1 and "limits" in str(ei.value)
