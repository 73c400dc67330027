"""CPU oracle for RECEIPT tip decomposition -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA
library in ``paper_2010_08695_gb300`` and imports nothing from it.

The arithmetic lives in ``oracle.c`` (plain C, compiled here with gcc and
OpenMP for the per-vertex counting loop only):

* ``count_2hop``   -- butterflies per vertex by their definition
  (sum over same-side x' of C(common neighbours, 2)), both sides;
* ``count_vp``     -- Algorithm 1 (pvBcnt), an independent cross-check;
* ``count_vertex`` -- the same definition for a list of vertices
  (``Graph.count_vertex`` on adjacency built once);
* ``bup``          -- Algorithm 2: sequential bottom-up peeling, with a
  monotone radix heap and the literal clamp of the support update.

``wing.c`` holds the edge analogue (wing decomposition, Sec. 7):

* ``edge_count``   -- butterflies of every edge by their definition;
* ``wing_bup``     -- sequential bottom-up edge peeling with the same clamp.

All functions take original-id edge lists ``(eu, ev)`` and return arrays
indexed by original id.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "wing.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc, -O2, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=199309L", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, *_SRCS]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class BupStats(ctypes.Structure):
    _fields_ = [("wedges", ctypes.c_uint64), ("peeled", ctypes.c_int64),
                ("seconds_count", ctypes.c_double), ("seconds_peel", ctypes.c_double),
                ("complete", ctypes.c_int64)]


class WingStats(ctypes.Structure):
    _fields_ = [("butterflies_visited", ctypes.c_uint64), ("edges_scanned", ctypes.c_uint64),
                ("peeled", ctypes.c_int64), ("complete", ctypes.c_int64)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        u64p = ctypes.c_void_p
        lib.oracle_count_2hop.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                          i32p, i32p, u64p, u64p]
        lib.oracle_count_vp.argtypes = lib.oracle_count_2hop.argtypes
        lib.oracle_count_vertex.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                            i32p, i32p, ctypes.c_int, i32p, ctypes.c_int64,
                                            u64p]
        lib.oracle_bup.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, i32p, i32p,
                                   ctypes.c_int, u64p, ctypes.c_uint64,
                                   ctypes.POINTER(BupStats)]
        lib.oracle_bup_from_counts.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                               i32p, i32p, ctypes.c_int, u64p, u64p,
                                               ctypes.c_uint64, ctypes.POINTER(BupStats)]
        lib.oracle_edge_count.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                          i32p, i32p, i32p, i32p, u64p,
                                          ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_wing_bup.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                        i32p, i32p, i32p, i32p, u64p,
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(WingStats)]
        lib.oracle_graph_new.restype = ctypes.c_void_p
        lib.oracle_graph_new.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, i32p,
                                         i32p, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_graph_count_vertex.argtypes = [ctypes.c_void_p, ctypes.c_int, i32p,
                                                  ctypes.c_int64, u64p,
                                                  ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_graph_free.argtypes = [ctypes.c_void_p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _prep(eu, ev):
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    if eu.shape != ev.shape:
        raise ValueError("eu and ev differ in length")
    return eu, ev


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise RuntimeError({1: "invalid input", 2: "out of memory"}.get(rc, f"rc={rc}"))


def count_2hop(eu, ev, nu, nv):
    """Per-vertex butterfly counts ``(cnt_u, cnt_v)`` by their definition."""
    eu, ev = _prep(eu, ev)
    cu = np.zeros(nu, np.uint64)
    cv = np.zeros(nv, np.uint64)
    _check(_load().oracle_count_2hop(nu, nv, len(eu), eu, ev, _ptr(cu), _ptr(cv)))
    return cu, cv


def count_vp(eu, ev, nu, nv):
    """Per-vertex butterfly counts ``(cnt_u, cnt_v)`` by Algorithm 1."""
    eu, ev = _prep(eu, ev)
    cu = np.zeros(nu, np.uint64)
    cv = np.zeros(nv, np.uint64)
    _check(_load().oracle_count_vp(nu, nv, len(eu), eu, ev, _ptr(cu), _ptr(cv)))
    return cu, cv


def count_vertex(eu, ev, nu, nv, side, xs):
    """Butterflies of the listed vertices of ``side`` (0 = U, 1 = V)."""
    eu, ev = _prep(eu, ev)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.zeros(len(xs), np.uint64)
    _check(_load().oracle_count_vertex(nu, nv, len(eu), eu, ev, int(side), xs, len(xs),
                                       _ptr(out)))
    return out


class Graph:
    """Adjacency of both sides built once, for repeated ``count_vertex``
    calls (e.g. a timed sample of vertices) without rebuilding it."""

    def __init__(self, eu, ev, nu, nv):
        eu, ev = _prep(eu, ev)
        rc = ctypes.c_int(0)
        self._h = _load().oracle_graph_new(nu, nv, len(eu), eu, ev, ctypes.byref(rc))
        _check(rc.value)
        self.nu, self.nv = nu, nv

    def count_vertex(self, side, xs):
        """``(counts, walked)``: butterflies of the listed vertices of ``side``
        and the 2-hop entries visited (sum over y in N_x of d_y)."""
        xs = np.ascontiguousarray(xs, dtype=np.int32)
        out = np.zeros(len(xs), np.uint64)
        walked = ctypes.c_uint64(0)
        _check(_load().oracle_graph_count_vertex(self._h, int(side), xs, len(xs), _ptr(out),
                                                 ctypes.byref(walked)))
        return out, int(walked.value)

    def close(self):
        if getattr(self, "_h", None):
            _load().oracle_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bup(eu, ev, nu, nv, side, max_wedges: int = 0):
    """Tip numbers of ``side`` by sequential bottom-up peeling.

    Returns ``(tips, stats)``; ``stats`` holds wedges traversed, vertices
    peeled, seconds of the initial count and of the peel, and whether the
    peel ran to completion (``max_wedges`` > 0 bounds it)."""
    eu, ev = _prep(eu, ev)
    n = nu if side == 0 else nv
    tips = np.zeros(n, np.uint64)
    st = BupStats()
    _check(_load().oracle_bup(nu, nv, len(eu), eu, ev, int(side), _ptr(tips),
                              int(max_wedges), ctypes.byref(st)))
    return tips, {"wedges": int(st.wedges), "peeled": int(st.peeled),
                  "seconds_count": st.seconds_count, "seconds_peel": st.seconds_peel,
                  "complete": bool(st.complete)}


def bup_from_counts(eu, ev, nu, nv, side, sup0, max_wedges: int = 0):
    """``bup`` started from given initial supports (the decomposed side's
    butterfly counts, e.g. from ``count_2hop``) instead of counting them."""
    eu, ev = _prep(eu, ev)
    n = nu if side == 0 else nv
    sup0 = np.ascontiguousarray(sup0, dtype=np.uint64)
    if len(sup0) != n:
        raise ValueError("sup0 has the wrong length")
    tips = np.zeros(n, np.uint64)
    st = BupStats()
    _check(_load().oracle_bup_from_counts(nu, nv, len(eu), eu, ev, int(side), _ptr(sup0),
                                          _ptr(tips), int(max_wedges), ctypes.byref(st)))
    return tips, {"wedges": int(st.wedges), "peeled": int(st.peeled),
                  "seconds_count": st.seconds_count, "seconds_peel": st.seconds_peel,
                  "complete": bool(st.complete)}


def edge_count(eu, ev, nu, nv):
    """Butterflies of every edge. Returns ``(eu, ev, cnt)`` over the
    duplicate-free edges in ascending ``(u, v)`` order."""
    eu, ev = _prep(eu, ev)
    ou = np.zeros(max(1, len(eu)), np.int32)
    ov = np.zeros(max(1, len(eu)), np.int32)
    cnt = np.zeros(max(1, len(eu)), np.uint64)
    mo = ctypes.c_int64(0)
    _check(_load().oracle_edge_count(nu, nv, len(eu), eu, ev, ou, ov, _ptr(cnt),
                                     ctypes.byref(mo)))
    k = mo.value
    return ou[:k], ov[:k], cnt[:k]


def wing_bup(eu, ev, nu, nv):
    """Wing numbers by sequential bottom-up edge peeling. Returns ``(eu, ev,
    wing, stats)`` over the duplicate-free edges in ascending ``(u, v)``
    order."""
    eu, ev = _prep(eu, ev)
    ou = np.zeros(max(1, len(eu)), np.int32)
    ov = np.zeros(max(1, len(eu)), np.int32)
    wing = np.zeros(max(1, len(eu)), np.uint64)
    mo = ctypes.c_int64(0)
    st = WingStats()
    _check(_load().oracle_wing_bup(nu, nv, len(eu), eu, ev, ou, ov, _ptr(wing),
                                   ctypes.byref(mo), ctypes.byref(st)))
    k = mo.value
    return ou[:k], ov[:k], wing[:k], {"butterflies": int(st.butterflies_visited),
                                      "edges_scanned": int(st.edges_scanned),
                                      "peeled": int(st.peeled),
                                      "complete": bool(st.complete)}


def num_threads() -> int:
    return int(_load().oracle_num_threads())
