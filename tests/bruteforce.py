"""Pure-Python brute force on tiny bipartite graphs, written from the
definitions only (no 2-hop counting formula, no peeling):

* a butterfly is a 2x2 biclique {u1, u2} x {v1, v2} (Sec. 2.1);
* the tip number of u is the largest k such that u lies in a k-tip, a
  subgraph induced on U' (with all of V) in which every vertex of U' takes
  part in at least k butterflies (Definition 1 and the text after it).

Connectivity and maximality in Definition 1 do not change the tip number:
the butterflies of u inside U' all lie in u's butterfly-connected component,
so that component alone is a k-tip whenever U' is. Hence
theta_u = max over subsets S containing u of min over z in S of the
butterflies of z inside S.
"""
from itertools import combinations


def butterflies(eu, ev):
    """All butterflies as tuples (u1, u2, v1, v2), u1 < u2, v1 < v2."""
    E = set(zip((int(a) for a in eu), (int(b) for b in ev)))
    U = sorted({u for u, _ in E})
    V = sorted({v for _, v in E})
    out = []
    for u1, u2 in combinations(U, 2):
        for v1, v2 in combinations(V, 2):
            if (u1, v1) in E and (u1, v2) in E and (u2, v1) in E and (u2, v2) in E:
                out.append((u1, u2, v1, v2))
    return out


def counts(eu, ev, nu, nv):
    """Per-vertex butterfly counts on both sides by enumeration."""
    cu = [0] * nu
    cv = [0] * nv
    for u1, u2, v1, v2 in butterflies(eu, ev):
        cu[u1] += 1
        cu[u2] += 1
        cv[v1] += 1
        cv[v2] += 1
    return cu, cv


def tip_numbers(eu, ev, nu, nv, side=0):
    """Tip numbers of ``side`` by maximising over all vertex subsets."""
    if side == 1:
        eu, ev, nu, nv = ev, eu, nv, nu
    bf = [(a, b) for a, b, _, _ in butterflies(eu, ev)]
    best = [0] * nu
    for mask in range(1, 1 << nu):
        sup = {}
        members = [x for x in range(nu) if mask >> x & 1]
        for x in members:
            sup[x] = 0
        for a, b in bf:
            if mask >> a & 1 and mask >> b & 1:
                sup[a] += 1
                sup[b] += 1
        k = min(sup.values())
        for x in members:
            if k > best[x]:
                best[x] = k
    return best


def edge_counts(eu, ev):
    """Butterflies containing each edge, by enumeration: {(u, v): count}."""
    E = set(zip((int(a) for a in eu), (int(b) for b in ev)))
    cnt = {e: 0 for e in E}
    for u1, u2, v1, v2 in butterflies(eu, ev):
        for e in ((u1, v1), (u1, v2), (u2, v1), (u2, v2)):
            cnt[e] += 1
    return cnt


def wing_numbers(eu, ev):
    """Wing numbers {(u, v): k} by maximising over all edge subsets H: the
    largest k such that e lies in some H whose every edge takes part in at
    least k butterflies of H (the edge analogue of Definition 1; as for tips,
    connectivity and maximality do not change the value). Tiny graphs only."""
    E = sorted(set(zip((int(a) for a in eu), (int(b) for b in ev))))
    idx = {e: i for i, e in enumerate(E)}
    bfs = [tuple(idx[e] for e in ((u1, v1), (u1, v2), (u2, v1), (u2, v2)))
           for u1, u2, v1, v2 in butterflies(eu, ev)]
    best = [0] * len(E)
    for mask in range(1, 1 << len(E)):
        sup = {i: 0 for i in range(len(E)) if mask >> i & 1}
        for b in bfs:
            if all(mask >> i & 1 for i in b):
                for i in b:
                    sup[i] += 1
        k = min(sup.values())
        for i in sup:
            if k > best[i]:
                best[i] = k
    return {e: best[i] for e, i in idx.items()}
