"""Pins of the CPU oracle to facts other than itself: brute-force enumeration
(butterflies as 2x2 bicliques; tip numbers as a maximum over vertex subsets,
Definition 1), closed forms on complete bipartite graphs, invariants (the sum
of per-vertex counts on each side is twice the number of butterflies; forests
hold no butterfly; tip number <= butterfly count), disjoint unions and the
U/V transposition."""
import numpy as np
import pytest

import oracle
import synth
from tests import bruteforce as bf


def _rand_graphs(n, max_u=8, max_v=7, seed=0):
    rng = np.random.default_rng(seed)
    for g in range(n):
        nu = int(rng.integers(1, max_u + 1))
        nv = int(rng.integers(1, max_v + 1))
        p = float(rng.uniform(0.2, 0.9))
        eu, ev = synth.random_small(nu, nv, p, int(rng.integers(1 << 30)))
        yield eu, ev, nu, nv


def test_counts_match_biclique_enumeration():
    for eu, ev, nu, nv in _rand_graphs(150, seed=1):
        cu, cv = oracle.count_2hop(eu, ev, nu, nv)
        bu, bv = bf.counts(eu, ev, nu, nv)
        assert cu.tolist() == bu
        assert cv.tolist() == bv


def test_vertex_priority_count_matches_enumeration():
    for eu, ev, nu, nv in _rand_graphs(150, seed=2):
        cu, cv = oracle.count_vp(eu, ev, nu, nv)
        bu, bv = bf.counts(eu, ev, nu, nv)
        assert cu.tolist() == bu
        assert cv.tolist() == bv


def test_sum_is_twice_butterflies():
    for eu, ev, nu, nv in _rand_graphs(60, max_u=9, max_v=9, seed=3):
        nb = len(bf.butterflies(eu, ev))
        cu, cv = oracle.count_2hop(eu, ev, nu, nv)
        assert int(cu.sum()) == 2 * nb
        assert int(cv.sum()) == 2 * nb


def test_tip_numbers_match_subset_definition():
    for side in (0, 1):
        for eu, ev, nu, nv in _rand_graphs(200, max_u=8, max_v=8, seed=10 + side):
            tips, st = oracle.bup(eu, ev, nu, nv, side)
            assert st["complete"]
            assert tips.tolist() == bf.tip_numbers(eu, ev, nu, nv, side)


@pytest.mark.parametrize("a,b", [(1, 1), (2, 2), (3, 5), (7, 4), (12, 9), (40, 3)])
def test_complete_bipartite_closed_form(a, b):
    eu, ev = synth.complete_bipartite(a, b)
    cu, cv = oracle.count_2hop(eu, ev, a, b)
    assert (cu == (a - 1) * (b * (b - 1) // 2)).all()
    assert (cv == (b - 1) * (a * (a - 1) // 2)).all()
    tu, _ = oracle.bup(eu, ev, a, b, 0)
    tv, _ = oracle.bup(eu, ev, a, b, 1)
    assert (tu == (a - 1) * (b * (b - 1) // 2)).all()
    assert (tv == (b - 1) * (a * (a - 1) // 2)).all()
    vu, vv = oracle.count_vp(eu, ev, a, b)
    assert (vu == cu).all() and (vv == cv).all()


def test_complete_bipartite_with_pendants():
    a, b = 6, 5
    eu, ev = synth.complete_bipartite(a, b)
    # pendant U vertices a..a+3 hang off V vertex 0; pendant V vertices b..b+2 off U 0
    eu = np.concatenate([eu, np.arange(a, a + 4, dtype=np.int32), np.zeros(3, np.int32)])
    ev = np.concatenate([ev, np.zeros(4, np.int32), np.arange(b, b + 3, dtype=np.int32)])
    nu, nv = a + 4, b + 3
    tu, _ = oracle.bup(eu, ev, nu, nv, 0)
    core = (a - 1) * (b * (b - 1) // 2)
    assert (tu[:a] == core).all() and (tu[a:] == 0).all()


def test_forests_have_no_butterflies():
    rng = np.random.default_rng(5)
    for _ in range(30):
        nu, nv = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        # random forest: each new vertex attaches to at most one earlier vertex
        eu, ev = [], []
        for v in range(1, nv):
            eu.append(int(rng.integers(nu)))
            ev.append(v)
        # make it a forest: every V vertex has degree 1
        eu, ev = np.array(eu, np.int32), np.array(ev, np.int32)
        cu, cv = oracle.count_2hop(eu, ev, nu, nv)
        assert cu.sum() == 0 and cv.sum() == 0
        t, _ = oracle.bup(eu, ev, nu, nv, 0)
        assert t.sum() == 0
    # a star
    eu = np.zeros(50, np.int32)
    ev = np.arange(50, dtype=np.int32)
    assert oracle.count_2hop(eu, ev, 1, 50)[1].sum() == 0


def test_disjoint_union_is_union_of_parts():
    rng = np.random.default_rng(7)
    parts = []
    for g in range(5):
        nu, nv = int(rng.integers(5, 60)), int(rng.integers(5, 40))
        m = int(rng.integers(1, nu * nv // 2 + 1))
        eu, ev = synth.er(nu, nv, m, int(rng.integers(1 << 30)))
        parts.append((eu, ev, nu, nv))
    ou = ov = 0
    EU, EV = [], []
    for eu, ev, nu, nv in parts:
        EU.append(eu + ou)
        EV.append(ev + ov)
        ou += nu
        ov += nv
    EU, EV = np.concatenate(EU), np.concatenate(EV)
    for side in (0, 1):
        whole, _ = oracle.bup(EU, EV, ou, ov, side)
        pieces = np.concatenate([oracle.bup(eu, ev, nu, nv, side)[0]
                                 for eu, ev, nu, nv in parts])
        assert (whole == pieces).all()


def test_transpose_symmetry():
    for seed in range(5):
        eu, ev = synth.er(80, 30, 700, seed)
        a, _ = oracle.bup(eu, ev, 80, 30, 1)
        b, _ = oracle.bup(ev, eu, 30, 80, 0)
        assert (a == b).all()
        cu, cv = oracle.count_2hop(eu, ev, 80, 30)
        tu, tv = oracle.count_2hop(ev, eu, 30, 80)
        assert (cu == tv).all() and (cv == tu).all()


def test_tip_bounded_by_count_and_counting_paths_agree():
    eu, ev, nu, nv, _ = synth.workload_graph(synth.ER_20K)
    cu, cv = oracle.count_2hop(eu, ev, nu, nv)
    vu, vv = oracle.count_vp(eu, ev, nu, nv)
    assert (cu == vu).all() and (cv == vv).all()
    for side, c in ((0, cu), (1, cv)):
        t, st = oracle.bup(eu, ev, nu, nv, side)
        assert st["complete"] and (t <= c).all()
    sample = np.array([0, 5, 17, 1999], np.int32)
    assert (oracle.count_vertex(eu, ev, nu, nv, 0, sample) == cu[sample]).all()


def test_chung_lu_counting_paths_agree():
    eu, ev = synth.chung_lu(3000, 800, 30000, 2.2, 2.4, seed=9)
    cu, cv = oracle.count_2hop(eu, ev, 3000, 800)
    vu, vv = oracle.count_vp(eu, ev, 3000, 800)
    assert (cu == vu).all() and (cv == vv).all()
    # listed vertices on adjacency built once: same counts, and the walk
    # visits sum_{y in N_x} d_y entries per vertex
    g = oracle.Graph(eu, ev, 3000, 800)
    du = np.bincount(eu, minlength=3000)
    dv = np.bincount(ev, minlength=800)
    for side, c, n in ((0, cu, 3000), (1, cv, 800)):
        xs = np.random.default_rng(side).choice(n, 50, replace=False).astype(np.int32)
        got, walked = g.count_vertex(side, xs)
        assert (got == c[xs]).all()
        a, b, d_o = (eu, ev, dv) if side == 0 else (ev, eu, du)
        assert walked == sum(int(d_o[b[a == x]].sum()) for x in xs)
    g.close()


def test_duplicates_and_edge_cases():
    eu = np.array([0, 0, 1, 1, 0, 1], np.int32)
    ev = np.array([0, 1, 0, 1, 0, 1], np.int32)  # K_{2,2} with two repeats
    cu, cv = oracle.count_2hop(eu, ev, 3, 2)
    assert cu.tolist() == [1, 1, 0] and cv.tolist() == [1, 1]
    t, _ = oracle.bup(eu, ev, 3, 2, 0)
    assert t.tolist() == [1, 1, 0]
    e = np.zeros(0, np.int32)
    assert oracle.bup(e, e, 4, 3, 0)[0].tolist() == [0, 0, 0, 0]
    assert oracle.bup(e, e, 0, 3, 0)[0].tolist() == []
    with pytest.raises(RuntimeError):
        oracle.count_2hop(np.array([5], np.int32), np.array([0], np.int32), 3, 2)


def test_bounded_peel_sample():
    eu, ev, nu, nv, _ = synth.workload_graph(synth.ER_20K)
    full, st_full = oracle.bup(eu, ev, nu, nv, 0)
    part, st = oracle.bup(eu, ev, nu, nv, 0, max_wedges=st_full["wedges"] // 3)
    assert not st["complete"] and 0 < st["peeled"] < nu
    assert st["wedges"] >= st_full["wedges"] // 3


def test_peel_from_given_counts_equals_full_bup():
    eu, ev = synth.chung_lu(3000, 700, 25000, 2.3, 2.2, seed=17)
    for side in (0, 1):
        full, _ = oracle.bup(eu, ev, 3000, 700, side)
        c = oracle.count_2hop(eu, ev, 3000, 700)[side]
        again, st = oracle.bup_from_counts(eu, ev, 3000, 700, side, c)
        assert st["complete"] and (again == full).all()


def test_stored_er_golden_reproduces():
    """The stored values of the 20k-edge workload are the oracle's: the same
    draw, the same count and tip digests (tests/golden/make_golden.py wrote
    them from synth and oracle only)."""
    import hashlib
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        synth.ER_20K + ".json")
    gold = json.load(open(path))
    eu, ev, nu, nv, side = synth.workload_graph(synth.ER_20K)
    assert synth.edges_sha256(eu, ev) == gold["edges_sha256"]

    def sha(a):
        return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()

    cu, cv = oracle.count_2hop(eu, ev, nu, nv)
    assert sha(cu) == gold["count_u_sha256"] and sha(cv) == gold["count_v_sha256"]
    t, _ = oracle.bup(eu, ev, nu, nv, side)
    assert sha(t) == gold["tips_sha256"]


def test_count_without_peeled_vertices_is_support_after_peeling():
    """The identity the recount of Sec. 4.1 rests on: after any set A of one
    side's vertices is peeled, a remaining vertex's raw support (its count
    minus the butterflies it shares with each vertex of A, Lemma 2) equals
    its butterfly count in the graph without A. Shared butterflies come from
    enumerated 2x2 bicliques; the count without A from the oracle."""
    rng = np.random.default_rng(41)
    for eu, ev, nu, nv in _rand_graphs(120, max_u=9, max_v=8, seed=42):
        bfs = bf.butterflies(eu, ev)
        for side in (0, 1):
            n = nu if side == 0 else nv
            A = set(int(a) for a in np.nonzero(rng.random(n) < 0.4)[0])
            full = bf.counts(eu, ev, nu, nv)[side]
            raw = list(full)
            for u1, u2, v1, v2 in bfs:
                p, q = (u1, u2) if side == 0 else (v1, v2)
                # a butterfly of two remaining vertices is never subtracted;
                # one with a peeled vertex is subtracted once from the other
                if p in A and q not in A:
                    raw[q] -= 1
                elif q in A and p not in A:
                    raw[p] -= 1
            ends = eu if side == 0 else ev
            keep = np.array([int(x) not in A for x in ends], dtype=bool)
            sub = oracle.count_2hop(eu[keep], ev[keep], nu, nv)[side]
            for x in range(n):
                if x not in A:
                    assert raw[x] == int(sub[x]), (side, x)


# ---------------------------------------------------------------------------
# Wing decomposition (edge peeling, Sec. 7): per-edge counts and wing numbers
# ---------------------------------------------------------------------------

def _as_dict(ou, ov, vals):
    return {(int(a), int(b)): int(c) for a, b, c in zip(ou, ov, vals)}


def test_edge_counts_match_biclique_enumeration():
    for eu, ev, nu, nv in _rand_graphs(150, max_u=9, max_v=8, seed=50):
        ou, ov, cnt = oracle.edge_count(eu, ev, nu, nv)
        assert _as_dict(ou, ov, cnt) == bf.edge_counts(eu, ev)


def test_edge_counts_sum_to_vertex_counts():
    """Each butterfly has four edges, two at each of its vertices: the edge
    counts sum to 4x the butterflies, and over a vertex's edges to twice the
    vertex's count."""
    for eu, ev, nu, nv in _rand_graphs(40, max_u=40, max_v=30, seed=51):
        ou, ov, cnt = oracle.edge_count(eu, ev, nu, nv)
        cu, cv = oracle.count_2hop(eu, ev, nu, nv)
        assert int(cnt.sum()) == 2 * int(cu.sum())
        su = np.bincount(ou, weights=cnt.astype(np.float64), minlength=nu)
        sv = np.bincount(ov, weights=cnt.astype(np.float64), minlength=nv)
        assert (su.astype(np.uint64) == 2 * cu).all()
        assert (sv.astype(np.uint64) == 2 * cv).all()


def test_wing_numbers_match_subset_definition():
    rng = np.random.default_rng(52)
    done = 0
    while done < 120:
        nu, nv = int(rng.integers(2, 6)), int(rng.integers(2, 6))
        eu, ev = synth.random_small(nu, nv, float(rng.uniform(0.4, 0.95)),
                                    int(rng.integers(1 << 30)))
        if len(set(zip(eu.tolist(), ev.tolist()))) > 13:
            continue
        ou, ov, wing, st = oracle.wing_bup(eu, ev, nu, nv)
        assert st["complete"] and st["peeled"] == len(ou)
        assert _as_dict(ou, ov, wing) == bf.wing_numbers(eu, ev)
        done += 1


@pytest.mark.parametrize("a,b", [(2, 2), (3, 5), (6, 4), (9, 2)])
def test_wing_complete_bipartite_and_pendants(a, b):
    eu, ev = synth.complete_bipartite(a, b)
    ou, ov, wing, _ = oracle.wing_bup(eu, ev, a, b)
    assert (wing == (a - 1) * (b - 1)).all()
    _, _, cnt = oracle.edge_count(eu, ev, a, b)
    assert (cnt == (a - 1) * (b - 1)).all()
    # pendant U vertices on V vertex 0 and pendant V vertices on U vertex 0
    eu2 = np.concatenate([eu, np.arange(a, a + 3, dtype=np.int32), np.zeros(2, np.int32)])
    ev2 = np.concatenate([ev, np.zeros(3, np.int32), np.arange(b, b + 2, dtype=np.int32)])
    ou, ov, wing, _ = oracle.wing_bup(eu2, ev2, a + 3, b + 2)
    core = (ou < a) & (ov < b)
    assert (wing[core] == (a - 1) * (b - 1)).all() and (wing[~core] == 0).all()


def test_wing_bounded_by_count_transpose_and_union():
    parts = []
    rng = np.random.default_rng(53)
    for g in range(4):
        nu, nv = int(rng.integers(5, 30)), int(rng.integers(5, 25))
        m = int(rng.integers(1, nu * nv // 2 + 1))
        eu, ev = synth.er(nu, nv, m, int(rng.integers(1 << 30)))
        parts.append((eu, ev, nu, nv))
        ou, ov, wing, _ = oracle.wing_bup(eu, ev, nu, nv)
        _, _, cnt = oracle.edge_count(eu, ev, nu, nv)
        assert (wing <= cnt).all()
        # transposed graph: same edges, same wing numbers
        tv, tu, twing, _ = oracle.wing_bup(ev, eu, nv, nu)
        assert _as_dict(ou, ov, wing) == _as_dict(tu, tv, twing)
    ou0 = ov0 = 0
    EU, EV, want = [], [], {}
    for eu, ev, nu, nv in parts:
        pu, pv, pw, _ = oracle.wing_bup(eu, ev, nu, nv)
        want.update({(int(a) + ou0, int(b) + ov0): int(c) for a, b, c in zip(pu, pv, pw)})
        EU.append(eu + ou0)
        EV.append(ev + ov0)
        ou0 += nu
        ov0 += nv
    wu, wv, ww, _ = oracle.wing_bup(np.concatenate(EU), np.concatenate(EV), ou0, ov0)
    assert _as_dict(wu, wv, ww) == want


def test_wing_forest_and_empty():
    eu = np.zeros(6, np.int32)
    ev = np.arange(6, dtype=np.int32)
    ou, ov, wing, st = oracle.wing_bup(eu, ev, 1, 6)
    assert len(ou) == 6 and (wing == 0).all() and st["butterflies"] == 0
    e = np.zeros(0, np.int32)
    ou, ov, wing, st = oracle.wing_bup(e, e, 3, 4)
    assert len(ou) == 0 and st["complete"]
