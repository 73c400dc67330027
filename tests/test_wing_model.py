"""Readings of Sec. 7 (RECEIPT carried over to edge peeling), checked on the
CPU with small sequential models against the wing oracle:

1. Peeling every remaining edge at the minimum level together is exact when
   a butterfly that loses several edges in one level is removed once, by
   its peeled edge with the smallest id (the priority order of edges).
2. The RECEIPT form is exact for any ranges: edges split by support into
   ranges peeled concurrently (coarse step, same rule), then each range's
   edges peeled exactly from their support at the range's start, with the
   edges of higher ranges kept as fixed context and those of lower ranges
   gone (fine step) -- the edge analogue of Theorems 1-2.

These models fix the design of a GPU path; they share nothing with the
CUDA library."""
import numpy as np

import oracle
import synth


def _prep(eu, ev):
    E = sorted(set(zip(eu.tolist(), ev.tolist())))
    eid = {e: i for i, e in enumerate(E)}
    Nu, Nv = {}, {}
    for u, v in E:
        Nu.setdefault(u, []).append(v)
        Nv.setdefault(v, []).append(u)
    return E, eid, Nu, Nv


def _butterflies(e, E, eid, Nu, Nv):
    """The other three edges of every butterfly {u, u'} x {v, v'} of e."""
    u, v = E[e]
    for up in Nv[v]:
        if up == u:
            continue
        for vp in Nu[u]:
            if vp != v and (up, vp) in eid:
                yield eid[(up, v)], eid[(u, vp)], eid[(up, vp)]


def _peel_level(F, live, s, E, eid, Nu, Nv):
    """One concurrent level: every butterfly of the peeled edges F whose
    edges are all live is removed once, by its smallest-id peeled edge."""
    inF = set(F)
    for e in F:
        for tri in _butterflies(e, E, eid, Nu, Nv):
            if not all(live(f) for f in tri):
                continue
            if any(f in inF and f < e for f in tri):
                continue
            for f in tri:
                if f not in inF and f in s:
                    s[f] -= 1


def level_synchronous(eu, ev):
    E, eid, Nu, Nv = _prep(eu, ev)
    s = {e: sum(1 for _ in _butterflies(e, E, eid, Nu, Nv)) for e in range(len(E))}
    wing, level = {}, 0
    while s:
        level = max(level, min(s.values()))
        F = [e for e in s if s[e] <= level]
        _peel_level(F, lambda f: f in s, s, E, eid, Nu, Nv)
        for e in F:
            wing[e] = level
            del s[e]
    return [wing[e] for e in range(len(E))]


def receipt_form(eu, ev, bounds):
    E, eid, Nu, Nv = _prep(eu, ev)
    m = len(E)
    sup = {e: sum(1 for _ in _butterflies(e, E, eid, Nu, Nv)) for e in range(m)}
    sub, init = [-1] * m, [0] * m
    for i, hi in enumerate(bounds):           # coarse step, range i
        for e in range(m):
            if sub[e] < 0:
                init[e] = sup[e]
        while True:
            F = [e for e in range(m) if sub[e] < 0 and sup[e] < hi]
            if not F:
                break
            rem = {e: sup[e] for e in range(m) if sub[e] < 0}
            _peel_level(F, lambda f: sub[f] < 0, rem, E, eid, Nu, Nv)
            sup.update(rem)
            for e in F:
                sub[e] = i
    P = len(bounds)
    for e in range(m):
        if sub[e] < 0:
            init[e], sub[e] = sup[e], P
    wing = [0] * m
    for i in range(P + 1):                    # fine step, one range at a time
        s = {e: init[e] for e in range(m) if sub[e] == i}
        level = 0
        while s:
            level = max(level, min(s.values()))
            F = [e for e in s if s[e] <= level]
            _peel_level(F, lambda f, i=i: sub[f] > i or f in s, s, E, eid, Nu, Nv)
            for e in F:
                wing[e] = level
                del s[e]
    return wing


def test_level_synchronous_peel_with_priority_is_exact():
    rng = np.random.default_rng(61)
    for _ in range(150):
        nu, nv = int(rng.integers(1, 12)), int(rng.integers(1, 12))
        eu, ev = synth.random_small(nu, nv, float(rng.uniform(0.2, 0.95)),
                                    int(rng.integers(1 << 30)))
        _, _, want, _ = oracle.wing_bup(eu, ev, nu, nv)
        assert level_synchronous(eu, ev) == [int(x) for x in want]


def test_receipt_form_is_exact_for_any_ranges():
    rng = np.random.default_rng(62)
    for _ in range(80):
        nu, nv = int(rng.integers(2, 11)), int(rng.integers(2, 11))
        eu, ev = synth.random_small(nu, nv, float(rng.uniform(0.3, 0.95)),
                                    int(rng.integers(1 << 30)))
        _, _, want, _ = oracle.wing_bup(eu, ev, nu, nv)
        top = int(want.max()) + 2 if len(want) else 2
        for _ in range(3):
            b = sorted({int(x) for x in rng.integers(1, top + 1, size=int(rng.integers(1, 6)))})
            assert receipt_form(eu, ev, b) == [int(x) for x in want], b
    eu, ev = synth.chung_lu(300, 100, 1800, 2.2, 2.1, seed=4)
    _, _, want, _ = oracle.wing_bup(eu, ev, 300, 100)
    for b in ([2], [1, 5, 20], [3, 9, 27, 81]):
        assert receipt_form(eu, ev, b) == [int(x) for x in want], b
