"""GB300-native RECEIPT tip decomposition -- Python binding of libreceipt.so.

A thin ctypes layer over the C ABI of ``include/receipt.h``: it marshals
arguments (device pointers of torch tensors, the current CUDA stream) and
nothing else; every step of counting and peeling runs in the CUDA kernels of
``csrc/``. There is no CPU fallback: if the library is missing or fails to
load, every call raises.

Functions carry the C names (``receipt_build_csr``, ``receipt_count_butterflies``,
``receipt_tip_decompose``, ``receipt_decompose_batch``,
``receipt_tip_decompose_host``, ``receipt_get_stats``, ``receipt_last_error``);
``Graph`` wraps the opaque graph handle.

Counts and tip numbers are exact unsigned 64-bit integers. They are returned
in ``torch.int64`` tensors holding the same bits (every value a graph of
fewer than 2^31 edges can produce is below 2^63).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libreceipt.so")
_lib = None
_lock = threading.Lock()

RECEIPT_OK = 0
_STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "OVERFLOW", 6: "BUSY",
           7: "INTERNAL"}
SIDE_U, SIDE_V = 0, 1


class ReceiptError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"receipt error {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("h_bounds", ctypes.POINTER(ctypes.c_uint64)),
                ("n_bounds", ctypes.c_int32), ("d_subset", ctypes.c_void_p),
                ("h_bounds_out", ctypes.POINTER(ctypes.c_uint64)), ("h_bounds_cap", ctypes.c_int32),
                ("h_p_eff", ctypes.POINTER(ctypes.c_int32)), ("timing", ctypes.c_int32),
                ("warp_max_w", ctypes.c_int32), ("slice_min_w", ctypes.c_int32),
                ("no_dgm", ctypes.c_int32), ("dgm_frac_1024", ctypes.c_int32),
                ("fd_heavy_w", ctypes.c_int64), ("round_graphs", ctypes.c_int32),
                ("huc", ctypes.c_int32), ("huc_factor_1024", ctypes.c_int32),
                ("slice_ctas", ctypes.c_int32), ("scan_frontier", ctypes.c_int32),
                ("fd_huc", ctypes.c_int32), ("range_max_n", ctypes.c_int32),
                ("slice_fetch", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("wedges_count", ctypes.c_uint64), ("wedges_cd", ctypes.c_uint64),
                ("wedges_fd", ctypes.c_uint64), ("wedges_bup", ctypes.c_uint64),
                ("rounds_cd", ctypes.c_int64), ("levels_fd", ctypes.c_int64),
                ("p_eff", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms_csr", ctypes.c_float), ("ms_count", ctypes.c_float), ("ms_cd", ctypes.c_float),
                ("ms_fd", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("peel_wedges", ctypes.c_uint64 * 5), ("peel_mids", ctypes.c_uint64 * 5),
                ("peel_anchors", ctypes.c_uint64 * 5), ("peel_launches", ctypes.c_int64 * 5),
                ("ms_peel", ctypes.c_float * 5), ("ms_fd_max_subset", ctypes.c_float),
                ("fd_max_subset_n", ctypes.c_int32), ("fd_max_subset_levels", ctypes.c_int64),
                ("fd_heavy_subsets", ctypes.c_int32), ("ms_fd_heavy", ctypes.c_float),
                ("levels_fd_heavy", ctypes.c_int64), ("fd_tasks", ctypes.c_int32),
                ("huc_recounts", ctypes.c_int32), ("wedges_recount", ctypes.c_uint64),
                ("cost_recount", ctypes.c_uint64), ("ms_recount", ctypes.c_float),
                ("fd_split_levels", ctypes.c_int32), ("peel_pairs", ctypes.c_uint64 * 5),
                ("count_points", ctypes.c_int64 * 5), ("fd_recounts", ctypes.c_int64),
                ("wedges_fd_recount", ctypes.c_uint64)]


class Round(ctypes.Structure):
    _fields_ = [("range", ctypes.c_int32), ("frontier", ctypes.c_int32), ("hi", ctypes.c_uint64),
                ("anchors", ctypes.c_uint64 * 5), ("wedges", ctypes.c_uint64 * 5),
                ("ms", ctypes.c_float * 5), ("recount", ctypes.c_int32)]


class Subset(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("heavy", ctypes.c_int32), ("levels", ctypes.c_int64),
                ("wedges_est", ctypes.c_uint64), ("ms", ctypes.c_float), ("pad", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int32), ("P", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_int64), ("batch_max_edges", ctypes.c_int32),
                ("batch_max_graphs", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("packed_requests", ctypes.c_int64), ("peak_inflight", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("peak_inflight_bytes", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("graphs_per_s", ctypes.c_double)]


def lib_path() -> str:
    return _LIB_PATH


def load(build_if_missing: bool = True):
    """Loads libreceipt.so (building it with nvcc first if it is missing or
    older than its sources). Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import _build
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.receipt_build_csr.argtypes = [vp, vp, i64, i32, i32, ctypes.c_int, vp,
                                          ctypes.POINTER(vp)]
        lib.receipt_graph_destroy.argtypes = [vp]
        lib.receipt_graph_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                           ctypes.POINTER(i64)]
        lib.receipt_count_butterflies.argtypes = [vp, vp, vp, vp]
        lib.receipt_graph_max_degree.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.receipt_graph_max_degree.restype = ctypes.c_int
        lib.receipt_count_butterflies_noalloc.argtypes = [vp, vp, vp, vp]
        lib.receipt_count_butterflies_noalloc.restype = ctypes.c_int
        lib.receipt_tip_decompose.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(Options), vp]
        lib.receipt_decompose_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int),
                                                i32, ctypes.POINTER(vp), ctypes.POINTER(Options), vp]
        lib.receipt_tip_decompose_host.argtypes = [vp, vp, i64, i32, i32, ctypes.c_int, vp,
                                                   ctypes.POINTER(Options), vp]
        lib.receipt_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        lib.receipt_last_error.restype = ctypes.c_char_p
        lib.receipt_options_default.argtypes = [ctypes.POINTER(Options)]
        lib.receipt_kernel_launches.restype = ctypes.c_uint64
        lib.receipt_get_trace.argtypes = [vp, ctypes.POINTER(Round), i32, ctypes.POINTER(i32)]
        lib.receipt_get_trace.restype = ctypes.c_int
        lib.receipt_get_subsets.argtypes = [vp, ctypes.POINTER(Subset), i32, ctypes.POINTER(i32)]
        lib.receipt_get_subsets.restype = ctypes.c_int
        lib.receipt_server_config_default.argtypes = [ctypes.POINTER(ServerConfig)]
        lib.receipt_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
        lib.receipt_server_submit.argtypes = [vp, vp, vp, i64, i32, i32, ctypes.c_int, vp,
                                              ctypes.POINTER(i64)]
        lib.receipt_server_wait.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(i32),
                                            ctypes.POINTER(ctypes.c_double)]
        lib.receipt_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        lib.receipt_server_destroy.argtypes = [vp]
        lib.receipt_support_bound.argtypes = [i64, i32, i32, i64,
                                              ctypes.POINTER(ctypes.c_uint64)]
        lib.receipt_support_bound.restype = ctypes.c_int
        for f in ("receipt_server_create", "receipt_server_submit", "receipt_server_wait",
                  "receipt_server_get_stats", "receipt_server_destroy"):
            getattr(lib, f).restype = ctypes.c_int
        for f in ("receipt_build_csr", "receipt_graph_destroy", "receipt_graph_info",
                  "receipt_count_butterflies", "receipt_tip_decompose",
                  "receipt_decompose_batch", "receipt_tip_decompose_host", "receipt_get_stats"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def receipt_last_error() -> str:
    return load().receipt_last_error().decode()


def _check(rc):
    if rc != RECEIPT_OK:
        raise ReceiptError(rc, receipt_last_error())


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _options(P=150, bounds=None, subset=None, bounds_out=None, p_eff=None, timing=False,
             warp_max_w=0, slice_min_w=0, dgm=True, dgm_frac_1024=0, fd_heavy_w=0,
             round_graphs=False, huc=0, huc_factor_1024=0, slice_ctas=0, scan_frontier=0,
             fd_huc=0, range_max_n=0, slice_fetch=0):
    o = Options()
    load().receipt_options_default(ctypes.byref(o))
    o.P = int(P)
    o.slice_fetch = int(slice_fetch)
    o.fd_huc = int(fd_huc)
    o.range_max_n = int(range_max_n)
    o.slice_ctas = int(slice_ctas)
    o.scan_frontier = int(scan_frontier)
    o.huc = int(huc)
    o.huc_factor_1024 = int(huc_factor_1024)
    o.fd_heavy_w = int(fd_heavy_w)
    # True: one graph launch per round; False: device-driven rounds; -1:
    # separate launches per round
    o.round_graphs = -1 if round_graphs == -1 else (1 if round_graphs else 0)
    o.dgm_frac_1024 = int(dgm_frac_1024)
    o.no_dgm = 0 if dgm else 1
    o.warp_max_w = int(warp_max_w)
    o.slice_min_w = int(slice_min_w)
    keep = []
    if bounds is not None:
        b = np.ascontiguousarray(bounds, dtype=np.uint64)
        keep.append(b)
        o.h_bounds = b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        o.n_bounds = len(b)
    if subset is not None:
        o.d_subset = subset.data_ptr()
    if bounds_out is not None:
        o.h_bounds_out = bounds_out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        o.h_bounds_cap = len(bounds_out)
    if p_eff is not None:
        o.h_p_eff = ctypes.pointer(p_eff)
        keep.append(p_eff)
    o.timing = 1 if timing else 0
    return o, keep


def receipt_build_csr(eu, ev, nu: int, nv: int, dedup: bool = True, stream=None):
    """Builds a graph from device int32 edge tensors; returns the raw handle."""
    lib = load()
    h = ctypes.c_void_p()
    m = int(eu.numel())
    _check(lib.receipt_build_csr(_dptr(eu) if m else None, _dptr(ev) if m else None, m, int(nu),
                                 int(nv), 1 if dedup else 0, _stream_handle(stream),
                                 ctypes.byref(h)))
    return h


def receipt_count_butterflies(handle, cnt_u, cnt_v, stream=None):
    _check(load().receipt_count_butterflies(handle, _dptr(cnt_u), _dptr(cnt_v),
                                            _stream_handle(stream)))


def receipt_count_butterflies_noalloc(handle, cnt_u, cnt_v, stream=None):
    """Butterfly counts into caller tensors without any device allocation
    (graphs up to 65,536 vertices per side and 1,048,576 edges; calls that may
    overlap on the GPU must be serialised by the caller)."""
    _check(load().receipt_count_butterflies_noalloc(handle, _dptr(cnt_u), _dptr(cnt_v),
                                                    _stream_handle(stream)))


def receipt_tip_decompose(handle, side: int, tip, options=None, stream=None):
    o = options if options is not None else _options()[0]
    _check(load().receipt_tip_decompose(handle, int(side), _dptr(tip), ctypes.byref(o),
                                        _stream_handle(stream)))


def receipt_get_stats(handle) -> dict:
    st = Stats()
    _check(load().receipt_get_stats(handle, ctypes.byref(st)))
    out = {}
    for k, _ in Stats._fields_:
        if k.startswith("reserved"):
            continue
        v = getattr(st, k)
        out[k] = list(v) if hasattr(v, "__len__") else v
    return out


def receipt_get_trace(handle) -> list:
    """Per-round records of the last decomposition (coarse-grained step)."""
    lib = load()
    n = ctypes.c_int32(0)
    _check(lib.receipt_get_trace(handle, None, 0, ctypes.byref(n)))
    buf = (Round * max(1, n.value))()
    _check(lib.receipt_get_trace(handle, buf, n.value, ctypes.byref(n)))
    return [{"range": r.range, "frontier": r.frontier, "hi": r.hi, "anchors": list(r.anchors),
             "wedges": list(r.wedges), "ms": list(r.ms), "recount": r.recount}
            for r in buf[: n.value]]


def receipt_get_subsets(handle) -> list:
    """Per-subset records of the last decomposition (fine-grained step)."""
    lib = load()
    n = ctypes.c_int32(0)
    _check(lib.receipt_get_subsets(handle, None, 0, ctypes.byref(n)))
    buf = (Subset * max(1, n.value))()
    _check(lib.receipt_get_subsets(handle, buf, n.value, ctypes.byref(n)))
    return [{"n": r.n, "heavy": bool(r.heavy), "levels": r.levels, "wedges_est": r.wedges_est,
             "ms": r.ms} for r in buf[: n.value]]


def receipt_support_bound(n_side: int, max_deg_side: int, max_deg_other: int, m: int) -> int:
    """Upper bound of any vertex's butterfly count on a side of that shape
    (host arithmetic, no device needed). Raises ReceiptError with
    RECEIPT_ERR_OVERFLOW (5) when it reaches 2^63."""
    b = ctypes.c_uint64(0)
    _check(load().receipt_support_bound(int(n_side), int(max_deg_side), int(max_deg_other),
                                        int(m), ctypes.byref(b)))
    return int(b.value)


def receipt_kernel_launches() -> int:
    """Kernels launched by libreceipt in this process so far."""
    return int(load().receipt_kernel_launches())


class Graph:
    """Device graph (relabelled two-sided CSR) owned by libreceipt."""

    def __init__(self, eu, ev, nu: int, nv: int, dedup: bool = True, stream=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        eu = torch.as_tensor(eu).to(device=dev, dtype=torch.int32).contiguous()
        ev = torch.as_tensor(ev).to(device=dev, dtype=torch.int32).contiguous()
        self.nu, self.nv = int(nu), int(nv)
        self.device = dev
        self._h = receipt_build_csr(eu, ev, nu, nv, dedup, stream)
        nu_, nv_, m_ = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(load().receipt_graph_info(self._h, ctypes.byref(nu_), ctypes.byref(nv_),
                                         ctypes.byref(m_)))
        self.m = int(m_.value)
        du, dv = ctypes.c_int32(), ctypes.c_int32()
        _check(load().receipt_graph_max_degree(self._h, ctypes.byref(du), ctypes.byref(dv)))
        self.max_degree = (int(du.value), int(dv.value))

    def shape_class(self, side: int) -> str:
        """Key of this graph in the autotuner's table."""
        from . import autotune
        return autotune.shape_class(self.nu, self.nv, self.m, side, self.max_degree[1 - side])

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().receipt_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def count_butterflies(self, stream=None):
        """Per-vertex butterfly counts ``(cnt_u, cnt_v)`` (Algorithm 1)."""
        import torch
        cu = torch.empty(self.nu, dtype=torch.int64, device=self.device)
        cv = torch.empty(self.nv, dtype=torch.int64, device=self.device)
        receipt_count_butterflies(self._h, cu, cv, stream)
        return cu, cv

    def tip_decompose(self, side: int = SIDE_U, P: int = 0, bounds=None, subsets=False,
                      timing=False, out=None, stream=None, warp_max_w=0, slice_min_w=0, dgm=True,
                      dgm_frac_1024=0, fd_heavy_w=0, round_graphs=False, huc=0,
                      huc_factor_1024=0, slice_ctas=0, scan_frontier=None, fd_huc=0,
                      range_max_n=None, slice_fetch=0):
        """Tip numbers of ``side`` (Algorithms 3 and 4). P = 0 takes the tuned
        value for this graph's shape class, else 150. With ``subsets=True``
        returns ``(tips, subset_of_vertex, range_bounds)``. ``huc``: 0 = the
        recount rule of Sec. 4.1, -1 = never recount, 1 = recount the first
        round of every range."""
        import torch
        n = self.nu if side == SIDE_U else self.nv
        tuned = None
        if not (warp_max_w and slice_min_w and P):
            from . import autotune
            tuned = autotune.lookup(self.shape_class(side))
        if tuned:
            warp_max_w = warp_max_w or tuned["warp_max_w"]
            slice_min_w = slice_min_w or tuned["slice_min_w"]
            P = P or tuned.get("P", 150)
            dgm_frac_1024 = dgm_frac_1024 or tuned.get("dgm_frac_1024", 0)
            slice_ctas = slice_ctas or tuned.get("slice_ctas", 0)
            if scan_frontier is None:
                scan_frontier = tuned.get("scan_frontier", 0)
            if range_max_n is None:
                range_max_n = _tuned_cap(tuned, P)
            slice_fetch = slice_fetch or tuned.get("slice_fetch", 0)
        P = P or 150
        tip = out if out is not None else torch.empty(n, dtype=torch.int64, device=self.device)
        sub = torch.empty(n, dtype=torch.int32, device=self.device) if subsets else None
        bout = np.zeros(P + (len(bounds) if bounds is not None else 0) + 4, np.uint64) \
            if subsets else None
        peff = ctypes.c_int32(0)
        o, keep = _options(P, bounds, sub, bout, peff, timing, warp_max_w, slice_min_w, dgm,
                           dgm_frac_1024, fd_heavy_w, round_graphs, huc, huc_factor_1024,
                           slice_ctas, int(scan_frontier or 0), fd_huc, int(range_max_n or 0),
                           slice_fetch)
        receipt_tip_decompose(self._h, side, tip, o, stream)
        if subsets:
            return tip, sub, bout[: peff.value + 1]
        return tip

    def stats(self) -> dict:
        return receipt_get_stats(self._h)

    def trace(self) -> list:
        return receipt_get_trace(self._h)

    def subsets(self) -> list:
        return receipt_get_subsets(self._h)


def _tuned_cap(rec, P):
    """The tuned vertex cap of a range for a run with P ranges: the table's
    cap was tuned with its own P, so the cap keeps cap * P (the vertices the
    capped ranges can hold together) when P differs; -1 (no cap) and 0
    (2 n / P) stay."""
    cap = int(rec.get("range_max_n", 0))
    tp = int(rec.get("P", 0))
    if cap > 0 and tp > 0 and P > 0 and P != tp:
        return max(1, (cap * tp + P // 2) // P)
    return cap


def receipt_decompose_batch(graphs, sides, outs=None, P: int = 0, stream=None, timing=False,
                            round_graphs=False, huc=0, huc_factor_1024=0, tuned=True, **options):
    """Tip numbers of many graphs in one pass (disjoint-union packing). With
    `tuned`, options not given take the autotuner's values for the union's
    shape class (P = 0: tuned, else 150)."""
    import torch
    n = len(graphs)
    if tuned and n > 0:
        from . import autotune
        rec = autotune.lookup(autotune.batch_shape_class(graphs, sides)) or {}
        for k in ("warp_max_w", "slice_min_w", "dgm_frac_1024", "slice_ctas", "slice_fetch"):
            if k in rec and not options.get(k):
                options[k] = rec[k]
        P = P or rec.get("P", 0)
        if rec and not options.get("range_max_n"):
            options["range_max_n"] = _tuned_cap(rec, P or 150)
    P = P or 150
    hs = (ctypes.c_void_p * n)(*[g.handle for g in graphs])
    ss = (ctypes.c_int * n)(*[int(s) for s in sides])
    if outs is None:
        outs = [torch.empty(g.nu if s == 0 else g.nv, dtype=torch.int64, device=g.device)
                for g, s in zip(graphs, sides)]
    ps = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    o, keep = _options(P, timing=timing, round_graphs=round_graphs, huc=huc,
                       huc_factor_1024=huc_factor_1024, **options)
    _check(load().receipt_decompose_batch(hs, ss, n, ps, ctypes.byref(o), _stream_handle(stream)))
    return outs


def receipt_tip_decompose_host(eu, ev, nu: int, nv: int, side: int, P: int = 150, stream=None,
                               out=None, **options):
    """End to end over host buffers: copies in, builds, decomposes, copies out.
    ``options`` are the keyword options of ``Graph.tip_decompose`` that only
    change speed (warp_max_w, slice_min_w, dgm, dgm_frac_1024, fd_heavy_w,
    round_graphs, huc, huc_factor_1024)."""
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    n = nu if side == SIDE_U else nv
    tip = out if out is not None else np.zeros(n, np.uint64)
    o, keep = _options(P, **options)
    _check(load().receipt_tip_decompose_host(eu.ctypes.data_as(ctypes.c_void_p),
                                             ev.ctypes.data_as(ctypes.c_void_p), len(eu), int(nu),
                                             int(nv), int(side), tip.ctypes.data_as(ctypes.c_void_p),
                                             ctypes.byref(o), _stream_handle(stream)))
    return tip


def as_u64(t) -> np.ndarray:
    """Device int64 tensor of exact counts -> host numpy uint64 (same bits)."""
    return t.cpu().numpy().view(np.uint64)


class Server:
    """Continuous-batching serving engine (receipt_server_*): submit host
    edge lists as requests arrive, wait for their tip numbers."""

    def __init__(self, max_inflight=4, P=150, mem_budget_bytes=0, batch_max_edges=200000,
                 batch_max_graphs=64):
        lib = load()
        cfg = ServerConfig()
        lib.receipt_server_config_default(ctypes.byref(cfg))
        cfg.max_inflight, cfg.P = int(max_inflight), int(P)
        cfg.mem_budget_bytes = int(mem_budget_bytes)
        cfg.batch_max_edges, cfg.batch_max_graphs = int(batch_max_edges), int(batch_max_graphs)
        self._h = ctypes.c_void_p()
        _check(lib.receipt_server_create(ctypes.byref(cfg), ctypes.byref(self._h)))
        self._keep = {}

    def submit(self, eu, ev, nu: int, nv: int, side: int):
        """Queues a decomposition; returns (request id, host output array)."""
        eu = np.ascontiguousarray(eu, dtype=np.int32)
        ev = np.ascontiguousarray(ev, dtype=np.int32)
        out = np.zeros(nu if side == SIDE_U else nv, np.uint64)
        rid = ctypes.c_int64()
        _check(load().receipt_server_submit(self._h, eu.ctypes.data_as(ctypes.c_void_p),
                                            ev.ctypes.data_as(ctypes.c_void_p), len(eu), int(nu),
                                            int(nv), int(side),
                                            out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rid)))
        self._keep[rid.value] = (eu, ev, out)
        return rid.value, out

    def wait(self, rid: int, timeout_s: float = 0.0):
        """Waits for a request; returns (tips, latency_ms). Raises on failure."""
        st = ctypes.c_int32()
        lat = ctypes.c_double()
        _check(load().receipt_server_wait(self._h, int(rid), float(timeout_s), ctypes.byref(st),
                                          ctypes.byref(lat)))
        eu, ev, out = self._keep.pop(rid)
        if st.value != RECEIPT_OK:
            raise ReceiptError(st.value, receipt_last_error())
        return out, lat.value

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().receipt_server_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_ if k != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            load().receipt_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
