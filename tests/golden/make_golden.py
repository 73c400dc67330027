"""Writes the stored expected values of the large parity cases.

Calls only ``synth`` (the seeded inputs) and ``oracle`` (the CPU reference);
nothing here touches the CUDA library. For each workload it records the
SHA-256 of the generated edge list (so a different draw on another machine is
caught before any comparison), the SHA-256 of the oracle's per-vertex
butterfly counts on both sides and of its tip numbers for the decomposed
side, plus a seeded sample of individual values for readable failures.

Usage: python tests/golden/make_golden.py [--vp-counts] WORKLOAD [WORKLOAD ...]
(workload names as in synth.WORKLOADS; each is written to tests/golden/<name>.json)

--vp-counts takes the initial supports from Algorithm 1 instead of the 2-hop
definition, after checking them against the 2-hop digests already stored for
the same graph (for the 100M-edge workload, whose 2-hop count alone takes most
of an hour).
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


def make(name, with_tips=True, vp_counts=False):
    t0 = time.time()
    eu, ev, nu, nv, side = synth.workload_graph(name)
    rec = {"workload": name, "nu": nu, "nv": nv, "m": int(len(eu)), "side": side,
           "edges_sha256": synth.edges_sha256(eu, ev)}
    t1 = time.time()
    if vp_counts:
        # Algorithm 1 (independent of the 2-hop definition, much faster); the
        # digests must equal the stored 2-hop ones of the same graph
        old = json.load(open(os.path.join(HERE, f"{name}.json")))
        assert old["edges_sha256"] == rec["edges_sha256"], "a different graph was drawn"
        cu, cv = oracle.count_vp(eu, ev, nu, nv)
        assert sha(cu) == old["count_u_sha256"] and sha(cv) == old["count_v_sha256"], \
            "Algorithm 1 and the 2-hop definition disagree"
        rec["seconds_count_2hop"] = old["seconds_count_2hop"]
        rec["seconds_count_vp"] = time.time() - t1
    else:
        cu, cv = oracle.count_2hop(eu, ev, nu, nv)
        rec["seconds_count_2hop"] = time.time() - t1
    rec["count_u_sha256"] = sha(cu)
    rec["count_v_sha256"] = sha(cv)
    rec["butterflies"] = int(cu.sum()) // 2
    rng = np.random.default_rng(1234 + synth.WORKLOADS[name]["seed"])
    su = np.unique(rng.integers(0, nu, 64))
    sv = np.unique(rng.integers(0, nv, 64))
    rec["sample_u"] = {int(x): int(cu[x]) for x in su}
    rec["sample_v"] = {int(x): int(cv[x]) for x in sv}
    rec["oracle_threads"] = oracle.num_threads()
    _write(name, rec)  # counts first: the peel of the largest workload takes hours
    if with_tips:
        # peel from the decomposed side's counts computed above
        tips, st = oracle.bup_from_counts(eu, ev, nu, nv, side, cu if side == 0 else cv)
        st["seconds_count"] = rec["seconds_count_2hop"]
        assert st["complete"]
        rec["tips_sha256"] = sha(tips)
        rec["tip_max"] = int(tips.max()) if len(tips) else 0
        rec["bup_wedges"] = st["wedges"]
        ss = su if side == 0 else sv
        rec["sample_tips"] = {int(x): int(tips[x]) for x in ss}
        rec["oracle_seconds"] = {"count": st["seconds_count"], "peel": st["seconds_peel"]}
    rec["wall_seconds"] = time.time() - t0
    _write(name, rec)
    print(json.dumps({k: rec[k] for k in rec if not k.startswith("sample")}))


def _write(name, rec):
    path = os.path.join(HERE, f"{name}.json")
    with open(path + ".tmp", "w") as f:
        json.dump(rec, f, indent=1, sort_keys=True)
    os.replace(path + ".tmp", path)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    for a in args:
        make(a, vp_counts="--vp-counts" in sys.argv)
