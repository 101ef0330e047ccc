"""GB300 Pregel superstep library: thin Python binding over ``libipg.so``.

The C ABI is declared in ``include/ipg.h``; every function here has the same name
as the C entry point it calls and only marshals arguments (numpy arrays for host
buffers, torch CUDA tensors for device buffers, a torch stream for ``*_dev``
calls).  All of the computation runs in the library's CUDA kernels; there is no
CPU fallback.  If the library has not been built, importing a function that needs
it raises ``IpgLibraryMissing``; build it with ``__graft_entry__.build()`` or
``paper_2010_01542_gb300._build.build()``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from ._build import library_path

__all__ = [
    "IpgError", "IpgLibraryMissing", "SuperstepStats", "Graph", "ipg_graph_create", "ipg_graph_create_dev",
    "ipg_graph_destroy", "ipg_graph_info", "ipg_graph_create_profile", "ipg_pagerank", "ipg_pagerank_dev", "ipg_hashmin_cc",
    "ipg_hashmin_cc_dev", "ipg_sssp", "ipg_sssp_dev", "ipg_last_error", "ipg_version",
    "IPG_STAT_RECEIVERS", "IPG_STAT_TIMING", "IPG_STAT_PULL", "INF", "load_library",
]

IPG_OK, IPG_EINVAL, IPG_ENOMEM, IPG_ECUDA, IPG_ETIMEOUT, IPG_EDEVICE, IPG_ENOTSUP, IPG_EOVERFLOW, IPG_ECANCELED = range(9)
STATUS_NAMES = ["IPG_OK", "IPG_EINVAL", "IPG_ENOMEM", "IPG_ECUDA", "IPG_ETIMEOUT", "IPG_EDEVICE", "IPG_ENOTSUP",
                "IPG_EOVERFLOW", "IPG_ECANCELED"]
IPG_STAT_RECEIVERS = 1
IPG_STAT_TIMING = 2
IPG_STAT_PULL = 4
INF = 0xFFFFFFFF


class IpgLibraryMissing(RuntimeError):
    pass


class IpgError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class _CStats(ctypes.Structure):
    _fields_ = [("superstep", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("active", ctypes.c_uint64),
                ("senders", ctypes.c_uint64), ("messages_sent", ctypes.c_uint64), ("receivers", ctypes.c_uint64),
                ("kernel_ms", ctypes.c_float), ("superstep_ms", ctypes.c_float)]


class _CStatsBuf(ctypes.Structure):
    _fields_ = [("buf", ctypes.POINTER(_CStats)), ("cap", ctypes.c_uint32), ("count", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


@dataclass
class SuperstepStats:
    superstep: int
    flags: int
    active: int
    senders: int
    messages_sent: int
    receivers: int
    kernel_ms: float
    superstep_ms: float


_lib = None


def load_library(path: Optional[str] = None):
    """Load libipg.so (once).  Raises IpgLibraryMissing if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise IpgLibraryMissing(f"{p} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    pstats = ctypes.POINTER(_CStatsBuf)
    lib.ipg_graph_create.argtypes = [vp, vp, vp, u32, u64, i32, ctypes.POINTER(vp)]
    lib.ipg_graph_create_dev.argtypes = [vp, vp, vp, u32, u64, i32, vp, ctypes.POINTER(vp)]
    lib.ipg_graph_destroy.argtypes = [vp]
    lib.ipg_graph_destroy.restype = None
    lib.ipg_graph_info.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(u64), ctypes.POINTER(i32),
                                   ctypes.POINTER(i32)]
    lib.ipg_pagerank.argtypes = [vp, u32, vp, pstats]
    lib.ipg_pagerank_dev.argtypes = [vp, u32, vp, pstats, vp]
    lib.ipg_hashmin_cc.argtypes = [vp, vp, pstats]
    lib.ipg_hashmin_cc_dev.argtypes = [vp, vp, pstats, vp]
    lib.ipg_sssp.argtypes = [vp, u32, vp, pstats]
    lib.ipg_sssp_dev.argtypes = [vp, u32, vp, pstats, vp]
    for f in ("ipg_graph_create", "ipg_graph_create_dev", "ipg_graph_info", "ipg_pagerank", "ipg_pagerank_dev",
              "ipg_hashmin_cc", "ipg_hashmin_cc_dev", "ipg_sssp", "ipg_sssp_dev"):
        getattr(lib, f).restype = i32
    lib.ipg_last_error.argtypes = []
    lib.ipg_last_error.restype = ctypes.c_char_p
    lib.ipg_status_string.argtypes = [i32]
    lib.ipg_status_string.restype = ctypes.c_char_p
    lib.ipg_version.argtypes = []
    lib.ipg_version.restype = i32
    if path is None:
        _lib = lib
    return lib


def ipg_last_error() -> str:
    return load_library().ipg_last_error().decode()


def ipg_version() -> int:
    return int(load_library().ipg_version())


def _check(rc: int):
    if rc != IPG_OK:
        raise IpgError(rc, ipg_last_error())


class Graph:
    """Owning handle for an ``ipg_graph*``; destroyed with the object or by ``ipg_graph_destroy``."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self):
        if not self._h:
            raise ValueError("graph has been destroyed")
        return self._h

    def destroy(self):
        if self._h:
            load_library().ipg_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def info(self):
        return ipg_graph_info(self)


def _host_ptr(a: Optional[np.ndarray], dtype, count: int, what: str):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=dtype)
    if a.size < count:
        raise ValueError(f"{what} has {a.size} entries, needs {count}")
    return a, (a.ctypes.data if a.size else None)


def ipg_graph_create(offsets, columns, weights, n: int, m: int, directed: bool) -> Graph:
    """Copy a host CSR graph (numpy arrays) to the current CUDA device."""
    lib = load_library()
    offs, po = _host_ptr(offsets, np.uint64, n + 1, "offsets")
    cols, pc = _host_ptr(columns, np.uint32, m, "columns")
    ws, pw = _host_ptr(weights, np.uint32, m, "weights")
    h = ctypes.c_void_p()
    _check(lib.ipg_graph_create(po, pc, pw, n, m, int(bool(directed)), ctypes.byref(h)))
    return Graph(h)


def _dev_ptr(t, itemsize: int, count: int, what: str):
    if t is None:
        return None
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous() or t.element_size() != itemsize:
        raise ValueError(f"{what} must be contiguous with {itemsize}-byte elements")
    if t.numel() < count:
        raise ValueError(f"{what} has {t.numel()} entries, needs {count}")
    return t.data_ptr() if count else None


def _stream_ptr(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def ipg_graph_create_dev(offsets, columns, weights, n: int, m: int, directed: bool, stream=None) -> Graph:
    """Copy a device CSR graph (torch CUDA tensors: 8-byte offsets, 4-byte columns/weights)."""
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.ipg_graph_create_dev(_dev_ptr(offsets, 8, n + 1, "offsets"), _dev_ptr(columns, 4, m, "columns"),
                                    _dev_ptr(weights, 4, m, "weights"), n, m, int(bool(directed)),
                                    _stream_ptr(stream), ctypes.byref(h)))
    return Graph(h)


def ipg_graph_destroy(g: Graph) -> None:
    g.destroy()


class _CCreateProfile(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("alloc_ms", "upload_issue_ms", "upload_ms", "validate_ms", "renumber_ms",
                                             "total_ms")]


def ipg_graph_create_profile(g: "Graph") -> dict:
    """Where ipg_graph_create spent its time, in milliseconds (see include/ipg.h)."""
    fn = load_library().ipg_graph_create_profile
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(_CCreateProfile)]
    fn.restype = ctypes.c_int
    p = _CCreateProfile()
    _check(fn(g.handle, ctypes.byref(p)))
    return {k: round(float(getattr(p, k)), 3) for k, _ in _CCreateProfile._fields_}


def ipg_graph_info(g: Graph):
    n, m, d, w = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().ipg_graph_info(g.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(d),
                                         ctypes.byref(w)))
    return {"n": n.value, "m": m.value, "directed": bool(d.value), "weighted": bool(w.value)}


def ipg_graph_check_symmetric(g: Graph, stream=None) -> bool:
    """True if the stored edges (with weights) equal their reverses: an undirected graph's check."""
    fn = _fn("ipg_graph_check_symmetric", [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p])
    sym = ctypes.c_int(-1)
    _check(fn(g.handle, ctypes.byref(sym), _stream_ptr(stream)))
    return bool(sym.value)


__all__ += ["ipg_graph_check_symmetric"]


class _Stats:
    def __init__(self, flags: int, cap: int):
        self.arr = (_CStats * max(cap, 1))()
        self.c = _CStatsBuf(ctypes.cast(self.arr, ctypes.POINTER(_CStats)), cap, 0, flags, 0)

    def result(self) -> List[SuperstepStats]:
        k = min(self.c.count, self.c.cap)
        return [SuperstepStats(int(s.superstep), int(s.flags), int(s.active), int(s.senders),
                               int(s.messages_sent), int(s.receivers), float(s.kernel_ms), float(s.superstep_ms))
                for s in self.arr[:k]]


def _run(fn, args, stats_flags: int, stats_cap: int):
    st = _Stats(stats_flags, stats_cap)
    _check(fn(*args, ctypes.byref(st.c)))
    return int(st.c.count), st.result()


def _run_dev(fn, args, stats_flags: int, stats_cap: int, stream):
    st = _Stats(stats_flags, stats_cap)
    _check(fn(*args, ctypes.byref(st.c), _stream_ptr(stream)))
    return int(st.c.count), st.result()


def ipg_pagerank(g: Graph, updates: int, ranks_out: Optional[np.ndarray] = None, stats_flags: int = 0,
                 stats_cap: int = 4096):
    """PageRank into a host float32 array.  Returns (ranks, supersteps, stats)."""
    n = ipg_graph_info(g)["n"]
    out = np.empty(n, dtype=np.float32) if ranks_out is None else ranks_out
    if out.dtype != np.float32 or not out.flags.c_contiguous or out.size < n:
        raise ValueError("ranks_out must be a contiguous float32 array of n entries")
    count, stats = _run(load_library().ipg_pagerank, (g.handle, updates, out.ctypes.data if n else None),
                        stats_flags, stats_cap)
    return out, count, stats


def ipg_pagerank_dev(g: Graph, updates: int, ranks_dev, stats_flags: int = 0, stats_cap: int = 4096, stream=None):
    """PageRank into a CUDA float32 tensor on `stream`.  Returns (supersteps, stats)."""
    n = ipg_graph_info(g)["n"]
    return _run_dev(load_library().ipg_pagerank_dev, (g.handle, updates, _dev_ptr(ranks_dev, 4, n, "ranks")),
                    stats_flags, stats_cap, stream)


def ipg_hashmin_cc(g: Graph, labels_out: Optional[np.ndarray] = None, stats_flags: int = 0, stats_cap: int = 1 << 16):
    """Hashmin components into a host uint32 array.  Returns (labels, supersteps, stats)."""
    n = ipg_graph_info(g)["n"]
    out = np.empty(n, dtype=np.uint32) if labels_out is None else labels_out
    if out.dtype != np.uint32 or not out.flags.c_contiguous or out.size < n:
        raise ValueError("labels_out must be a contiguous uint32 array of n entries")
    count, stats = _run(load_library().ipg_hashmin_cc, (g.handle, out.ctypes.data if n else None), stats_flags,
                        stats_cap)
    return out, count, stats


def ipg_hashmin_cc_dev(g: Graph, labels_dev, stats_flags: int = 0, stats_cap: int = 1 << 16, stream=None):
    n = ipg_graph_info(g)["n"]
    return _run_dev(load_library().ipg_hashmin_cc_dev, (g.handle, _dev_ptr(labels_dev, 4, n, "labels")),
                    stats_flags, stats_cap, stream)


def ipg_sssp(g: Graph, source: int, dist_out: Optional[np.ndarray] = None, stats_flags: int = 0,
             stats_cap: int = 1 << 16):
    """SSSP into a host uint32 array (INF = unreachable).  Returns (dist, supersteps, stats)."""
    n = ipg_graph_info(g)["n"]
    out = np.empty(n, dtype=np.uint32) if dist_out is None else dist_out
    if out.dtype != np.uint32 or not out.flags.c_contiguous or out.size < n:
        raise ValueError("dist_out must be a contiguous uint32 array of n entries")
    count, stats = _run(load_library().ipg_sssp, (g.handle, source, out.ctypes.data if n else None), stats_flags,
                        stats_cap)
    return out, count, stats


def ipg_sssp_dev(g: Graph, source: int, dist_dev, stats_flags: int = 0, stats_cap: int = 1 << 16, stream=None):
    n = ipg_graph_info(g)["n"]
    return _run_dev(load_library().ipg_sssp_dev, (g.handle, source, _dev_ptr(dist_dev, 4, n, "dist")),
                    stats_flags, stats_cap, stream)


def ipg_sssp_noalloc(offsets, columns, weights, n: int, m: int, source: int, dist_dev, stream=None) -> int:
    """SSSP on a caller-owned device CSR (torch CUDA tensors) into ``dist_dev``, with no
    device allocation by the library (fixed scratch, n <= IPG_NOALLOC_MAX_VERTICES).
    Returns the superstep count."""
    lib = load_library()
    fn = lib.ipg_sssp_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                   ctypes.c_uint32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    steps = ctypes.c_uint32()
    _check(fn(_dev_ptr(offsets, 8, n + 1, "offsets"), _dev_ptr(columns, 4, m, "columns"),
              _dev_ptr(weights, 4, m, "weights"), n, m, source, _dev_ptr(dist_dev, 4, n, "dist"),
              ctypes.byref(steps), _stream_ptr(stream)))
    return int(steps.value)


IPG_NOALLOC_MAX_VERTICES = 1 << 20
__all__ += ["ipg_sssp_noalloc", "IPG_NOALLOC_MAX_VERTICES"]


def ipg_set_tuning(name: str, value: int) -> None:
    """Set a process-wide tuning knob (see include/ipg.h); speed only, never results."""
    lib = load_library()
    lib.ipg_set_tuning.argtypes = [ctypes.c_char_p, ctypes.c_int64]
    lib.ipg_set_tuning.restype = ctypes.c_int
    _check(lib.ipg_set_tuning(name.encode(), int(value)))


def ipg_get_tuning(name: str) -> int:
    lib = load_library()
    lib.ipg_get_tuning.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64)]
    lib.ipg_get_tuning.restype = ctypes.c_int
    v = ctypes.c_int64()
    _check(lib.ipg_get_tuning(name.encode(), ctypes.byref(v)))
    return int(v.value)


__all__ += ["ipg_set_tuning", "ipg_get_tuning"]

IPG_TUNE_PAGERANK = 1
IPG_TUNE_HASHMIN = 2
IPG_TUNE_SSSP = 4
IPG_TUNE_SSSP_BATCH = 8
IPG_TUNE_FORCE = 0x100


class _CTuneReport(ctypes.Structure):
    _fields_ = [("programs", ctypes.c_uint32), ("cached", ctypes.c_uint32),
                ("hashmin_pull_divisor", ctypes.c_int64), ("sssp_pull_divisor", ctypes.c_int64),
                ("sssp_batch_divisor", ctypes.c_int64), ("pr_engine", ctypes.c_int64), ("pr_carveout", ctypes.c_int64),
                ("hashmin_ms", ctypes.c_float), ("sssp_ms", ctypes.c_float), ("sssp_batch_ms", ctypes.c_float),
                ("pagerank_ms", ctypes.c_float), ("hashmin_default_ms", ctypes.c_float),
                ("sssp_default_ms", ctypes.c_float), ("sssp_batch_default_ms", ctypes.c_float),
                ("pagerank_default_ms", ctypes.c_float), ("candidates_timed", ctypes.c_uint32),
                ("sssp_batch_chunk", ctypes.c_uint32)]


def ipg_autotune(g: Graph, programs: int, sssp_source: int = INF, stream=None) -> dict:
    """Tune the graph's launch shape by timing candidates on it (include/ipg.h); returns the report."""
    lib = load_library()
    lib.ipg_autotune.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_CTuneReport),
                                 ctypes.c_void_p]
    lib.ipg_autotune.restype = ctypes.c_int
    rep = _CTuneReport()
    _check(lib.ipg_autotune(g.handle, int(programs), int(sssp_source), ctypes.byref(rep), _stream_ptr(stream)))
    return {name: getattr(rep, name) for name, _ in _CTuneReport._fields_}


__all__ += ["ipg_autotune", "IPG_TUNE_PAGERANK", "IPG_TUNE_HASHMIN", "IPG_TUNE_SSSP", "IPG_TUNE_SSSP_BATCH",
            "IPG_TUNE_FORCE"]


def _sources_arr(sources, n):
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.uint32).ravel())
    return src


def ipg_sssp_batch(g: Graph, sources, dist_out: Optional[np.ndarray] = None):
    """k SSSP runs (one per source) together.  Returns (dist[k, n] uint32, supersteps[k])."""
    lib = load_library()
    n = ipg_graph_info(g)["n"]
    src = _sources_arr(sources, n)
    k = src.size
    out = np.empty((k, n), dtype=np.uint32) if dist_out is None else dist_out
    if out.dtype != np.uint32 or not out.flags.c_contiguous or out.size < k * n:
        raise ValueError("dist_out must be a contiguous uint32 array of k * n entries")
    steps = np.zeros(k, dtype=np.uint32)
    fn = lib.ipg_sssp_batch
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    _check(fn(g.handle, src.ctypes.data if k else None, k, out.ctypes.data if k * n else None,
              steps.ctypes.data if k else None))
    return out, steps


def ipg_sssp_batch_dev(g: Graph, sources, dist_dev, stream=None):
    """k SSSP runs into a CUDA tensor of k * n 4-byte entries (row i from sources[i]).
    Returns supersteps[k]."""
    lib = load_library()
    n = ipg_graph_info(g)["n"]
    src = _sources_arr(sources, n)
    k = src.size
    steps = np.zeros(k, dtype=np.uint32)
    fn = lib.ipg_sssp_batch_dev
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    _check(fn(g.handle, src.ctypes.data if k else None, k, _dev_ptr(dist_dev, 4, k * n, "dist"),
              steps.ctypes.data if k else None, _stream_ptr(stream)))
    return steps


__all__ += ["ipg_sssp_batch", "ipg_sssp_batch_dev", "ipg_sssp_batch_info"]


class _CBatchInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("queries", "supersteps", "pull_supersteps", "harvests", "launches", "lanes")]


def ipg_sssp_batch_info(g: "Graph") -> dict:
    """Totals of the graph's last batched SSSP call (see include/ipg.h)."""
    fn = load_library().ipg_sssp_batch_info
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(_CBatchInfo)]
    fn.restype = ctypes.c_int
    r = _CBatchInfo()
    _check(fn(g.handle, ctypes.byref(r)))
    return {k: int(getattr(r, k)) for k, _ in _CBatchInfo._fields_}


def ipg_graph_create_batch(graphs, directed: bool) -> Graph:
    """One graph object holding several independent host CSR graphs (objects with n,
    offsets, cols and optional weights).  Instance i's vertices follow instance i-1's."""
    lib = load_library()
    count = len(graphs)
    keep = []
    P64, P32 = ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)
    offs = (P64 * count)()
    cols = (P32 * count)()
    ws = (P32 * count)()
    ns = (ctypes.c_uint32 * count)()
    ms = (ctypes.c_uint64 * count)()
    weighted = count > 0 and all(getattr(gr, "weights", None) is not None for gr in graphs)
    for i, gr in enumerate(graphs):
        o = np.ascontiguousarray(gr.offsets, dtype=np.uint64)
        c = np.ascontiguousarray(gr.cols, dtype=np.uint32)
        keep += [o, c]
        offs[i] = o.ctypes.data_as(P64)
        cols[i] = c.ctypes.data_as(P32) if c.size else P32()
        if weighted:
            w = np.ascontiguousarray(gr.weights, dtype=np.uint32)
            keep.append(w)
            ws[i] = w.ctypes.data_as(P32) if w.size else P32()
        ns[i] = int(gr.n)
        ms[i] = int(o[-1])
    fn = lib.ipg_graph_create_batch
    fn.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    fn.restype = ctypes.c_int
    h = ctypes.c_void_p()
    _check(fn(count, offs, cols, ws if weighted else None, ns, ms, int(bool(directed)), ctypes.byref(h)))
    return Graph(h)


def ipg_graph_instances(g: Graph):
    """(count, bases[count + 1])"""
    lib = load_library()
    fn = lib.ipg_graph_instances
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    c = ctypes.c_uint32()
    _check(fn(g.handle, ctypes.byref(c), None))
    bases = np.zeros(c.value + 1, dtype=np.uint32)
    _check(fn(g.handle, ctypes.byref(c), bases.ctypes.data))
    return int(c.value), bases


def ipg_hashmin_cc_batch(g: Graph, labels_out: Optional[np.ndarray] = None):
    """Hashmin on every instance.  Returns (labels[total n] instance-local, supersteps[count])."""
    lib = load_library()
    n = ipg_graph_info(g)["n"]
    count, _ = ipg_graph_instances(g)
    out = np.empty(n, dtype=np.uint32) if labels_out is None else labels_out
    steps = np.zeros(count, dtype=np.uint32)
    fn = lib.ipg_hashmin_cc_batch
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    _check(fn(g.handle, out.ctypes.data if n else None, steps.ctypes.data))
    return out, steps


def ipg_hashmin_cc_batch_dev(g: Graph, labels_dev, stream=None):
    lib = load_library()
    n = ipg_graph_info(g)["n"]
    count, _ = ipg_graph_instances(g)
    steps = np.zeros(count, dtype=np.uint32)
    fn = lib.ipg_hashmin_cc_batch_dev
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    _check(fn(g.handle, _dev_ptr(labels_dev, 4, n, "labels"), steps.ctypes.data, _stream_ptr(stream)))
    return steps


__all__ += ["ipg_graph_create_batch", "ipg_graph_instances", "ipg_hashmin_cc_batch", "ipg_hashmin_cc_batch_dev"]


# ---------------------------------------------------------------------------------------
# general combiners (Sec. III, Fig. 1): wider messages through the hybrid combiner

IPG_COMBINE_XOR_U32, IPG_COMBINE_MIN_U64, IPG_COMBINE_SUM_U64, IPG_COMBINE_MINCOUNT_U128 = 0, 1, 2, 3
IPG_COMBINE_WARP = 1
IPG_COMBINE_NATIVE = 2
IPG_COMBINE_STALLED = 4
_COMBINE_SIZE = {IPG_COMBINE_XOR_U32: 4, IPG_COMBINE_MIN_U64: 8, IPG_COMBINE_SUM_U64: 8, IPG_COMBINE_MINCOUNT_U128: 16}


def _fn(name, argtypes):
    fn = getattr(load_library(), name)
    fn.argtypes = argtypes
    fn.restype = ctypes.c_int
    return fn


_VP, _U32, _U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
_PSTATS = ctypes.POINTER(_CStatsBuf)


def ipg_sssp_tree(g: Graph, source: int, stats_flags: int = 0, stats_cap: int = 1 << 16):
    """SSSP with its shortest-path tree into host arrays.  Returns (dist, parent, supersteps, stats)."""
    n = ipg_graph_info(g)["n"]
    dist = np.empty(n, dtype=np.uint32)
    parent = np.empty(n, dtype=np.uint32)
    fn = _fn("ipg_sssp_tree", [_VP, _U32, _VP, _VP, _PSTATS])
    count, stats = _run(fn, (g.handle, source, dist.ctypes.data if n else None, parent.ctypes.data if n else None),
                        stats_flags, stats_cap)
    return dist, parent, count, stats


def ipg_sssp_tree_dev(g: Graph, source: int, dist_dev, parent_dev, stats_flags: int = 0, stats_cap: int = 1 << 16,
                      stream=None):
    n = ipg_graph_info(g)["n"]
    fn = _fn("ipg_sssp_tree_dev", [_VP, _U32, _VP, _VP, _PSTATS, _VP])
    return _run_dev(fn, (g.handle, source, _dev_ptr(dist_dev, 4, n, "dist"), _dev_ptr(parent_dev, 4, n, "parent")),
                    stats_flags, stats_cap, stream)


def ipg_bfs_paths(g: Graph, source: int, stats_flags: int = 0, stats_cap: int = 1 << 16):
    """Shortest-path counts from `source` into host arrays.  Returns (level, paths, supersteps, stats)."""
    n = ipg_graph_info(g)["n"]
    level = np.empty(n, dtype=np.uint32)
    paths = np.empty(n, dtype=np.uint64)
    fn = _fn("ipg_bfs_paths", [_VP, _U32, _VP, _VP, _PSTATS])
    count, stats = _run(fn, (g.handle, source, level.ctypes.data if n else None, paths.ctypes.data if n else None),
                        stats_flags, stats_cap)
    return level, paths, count, stats


def ipg_bfs_paths_dev(g: Graph, source: int, level_dev, paths_dev, stats_flags: int = 0, stats_cap: int = 1 << 16,
                      stream=None):
    n = ipg_graph_info(g)["n"]
    fn = _fn("ipg_bfs_paths_dev", [_VP, _U32, _VP, _VP, _PSTATS, _VP])
    return _run_dev(fn, (g.handle, source, _dev_ptr(level_dev, 4, n, "level"), _dev_ptr(paths_dev, 8, n, "paths")),
                    stats_flags, stats_cap, stream)


def ipg_combine_dev(kind: int, n: int, dst_dev, msgs_dev, flags_dev, mail_dev, options: int = 0, stream=None) -> int:
    """Deliver messages msgs_dev[i] to dst_dev[i] into n empty mailboxes (CUDA tensors:
    dst int32/uint32 [k]; msgs of the kind's size — int32 [k], int64 [k] or int64 [k, 2];
    flags int32 [n]; mail like msgs with n rows).  Returns the number of receivers."""
    size = _COMBINE_SIZE.get(kind, 8)  # an unknown kind is left to the library to reject
    k = 0 if dst_dev is None else dst_dev.numel()
    width = 2 if size == 16 else 1
    esize = 4 if size == 4 else 8
    if msgs_dev is not None and msgs_dev.numel() < k * width:
        raise ValueError("msgs has fewer entries than dst")
    fn = _fn("ipg_combine_dev", [ctypes.c_int, _U32, _VP, _VP, _U64, _VP, _VP, ctypes.POINTER(_U64), _U32, _VP])
    recv = ctypes.c_uint64()
    _check(fn(kind, n, _dev_ptr(dst_dev, 4, k, "dst"), _dev_ptr(msgs_dev, esize, k * width, "msgs"), k,
              _dev_ptr(flags_dev, 4, n, "flags"), _dev_ptr(mail_dev, esize, n * width, "mail"), ctypes.byref(recv),
              options, _stream_ptr(stream)))
    return int(recv.value)


__all__ += ["ipg_sssp_tree", "ipg_sssp_tree_dev", "ipg_bfs_paths", "ipg_bfs_paths_dev", "ipg_combine_dev",
            "IPG_COMBINE_XOR_U32", "IPG_COMBINE_MIN_U64", "IPG_COMBINE_SUM_U64", "IPG_COMBINE_MINCOUNT_U128",
            "IPG_COMBINE_WARP", "IPG_COMBINE_NATIVE", "IPG_COMBINE_STALLED"]


# ---------------------------------------------------------------------------------------
# serving

IPG_Q_SSSP, IPG_Q_HASHMIN, IPG_Q_PAGERANK = 0, 1, 2


class _CQuery(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_uint32), ("kind", ctypes.c_uint32), ("source", ctypes.c_uint32),
                ("updates", ctypes.c_uint32), ("out", ctypes.c_void_p), ("user", ctypes.c_uint64)]


class _CCompletion(ctypes.Structure):
    _fields_ = [("user", ctypes.c_uint64), ("status", ctypes.c_int), ("supersteps", ctypes.c_uint32),
                ("batch", ctypes.c_uint32), ("joined", ctypes.c_uint32), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


IPG_SERVER_AUTOTUNE = 1
IPG_SERVER_PREPARE = 2


class _COptions(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_uint32), ("max_batch", ctypes.c_uint32), ("workspace_budget", ctypes.c_uint64),
                ("reserve_bytes", ctypes.c_uint64), ("min_sssp_batch", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


@dataclass
class Completion:
    user: int
    status: int
    supersteps: int
    batch: int
    t_submit: float
    t_start: float
    t_done: float
    out: Optional[np.ndarray] = None
    joined: int = 0  # 1: an SSSP query that joined a lane session already running on the device


class Server:
    """Binding of ipg_server_*: graphs stay resident, queries are served with continuous
    batching by the library's worker threads.  Output arrays are kept alive here until their
    completion is polled."""

    def __init__(self, graphs, workers: int = 0, max_batch: int = 0, workspace_budget: int = 0,
                 reserve_bytes: int = 0, min_sssp_batch: int = 0, autotune: bool = False,
                 prepare: bool = False):
        lib = load_library()
        self._lib = lib
        self._graphs = list(graphs)
        lib.ipg_server_create.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(_COptions),
                                          ctypes.POINTER(ctypes.c_void_p)]
        lib.ipg_server_create.restype = ctypes.c_int
        lib.ipg_server_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(_CQuery)]
        lib.ipg_server_submit.restype = ctypes.c_int
        lib.ipg_server_poll.argtypes = [ctypes.c_void_p, ctypes.POINTER(_CCompletion), ctypes.c_uint32, ctypes.c_int]
        lib.ipg_server_poll.restype = ctypes.c_uint32
        lib.ipg_server_cancel.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32)]
        lib.ipg_server_cancel.restype = ctypes.c_int
        lib.ipg_server_drain.argtypes = [ctypes.c_void_p]
        lib.ipg_server_drain.restype = ctypes.c_int
        lib.ipg_server_now.argtypes = [ctypes.c_void_p]
        lib.ipg_server_now.restype = ctypes.c_double
        lib.ipg_server_destroy.argtypes = [ctypes.c_void_p]
        lib.ipg_server_destroy.restype = None
        handles = (ctypes.c_void_p * len(self._graphs))(*[g.handle for g in self._graphs])
        opt = _COptions(workers, max_batch, workspace_budget, reserve_bytes, min_sssp_batch,
                        (IPG_SERVER_AUTOTUNE if autotune else 0) | (IPG_SERVER_PREPARE if prepare else 0))
        h = ctypes.c_void_p()
        _check(lib.ipg_server_create(handles, len(self._graphs), ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self._outs = {}
        self._buf = (_CCompletion * 1024)()

    def submit(self, graph: int, kind: int, out: np.ndarray, source: int = 0, updates: int = 10, user: int = 0):
        q = _CQuery(graph, kind, source, updates, out.ctypes.data if out.size else None, user)
        self._outs[user] = out
        try:
            _check(self._lib.ipg_server_submit(self._h, ctypes.byref(q)))
        except Exception:
            self._outs.pop(user, None)
            raise

    def poll(self, wait_ms: int = 0) -> List[Completion]:
        k = self._lib.ipg_server_poll(self._h, self._buf, len(self._buf), wait_ms)
        res = []
        for c in self._buf[:k]:
            res.append(Completion(int(c.user), int(c.status), int(c.supersteps), int(c.batch), float(c.t_submit),
                                  float(c.t_start), float(c.t_done), self._outs.pop(int(c.user), None),
                                  int(c.joined)))
        return res

    def cancel(self, user: int) -> int:
        """Cancel the queued, not yet dispatched queries tagged `user`; returns how many.
        Each still produces a completion (status IPG_ECANCELED) for poll()."""
        k = ctypes.c_uint32(0)
        _check(self._lib.ipg_server_cancel(self._h, user, ctypes.byref(k)))
        return int(k.value)

    def drain(self):
        _check(self._lib.ipg_server_drain(self._h))

    def now(self) -> float:
        return float(self._lib.ipg_server_now(self._h))

    def close(self):
        if self._h:
            self._lib.ipg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ += ["Server", "Completion", "IPG_Q_SSSP", "IPG_Q_HASHMIN", "IPG_Q_PAGERANK"]


class HostBuffer:
    """Page-locked host memory from ``ipg_host_alloc`` (huge-page backed where the kernel allows).

    Freed with ``ipg_host_free`` when the object goes away; numpy arrays made by
    ``host_empty`` keep it alive through their ``base``.
    """

    def __init__(self, nbytes: int):
        fn = _fn("ipg_host_alloc", [ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)])
        p = ctypes.c_void_p()
        _check(fn(int(nbytes), ctypes.byref(p)))
        self.ptr = p.value or 0
        self.nbytes = int(nbytes)

    @property
    def __array_interface__(self):
        return {"shape": (self.nbytes,), "typestr": "|u1", "data": (self.ptr, False), "version": 3}

    def free(self):
        if self.ptr:
            _fn("ipg_host_free", [ctypes.c_void_p])(ctypes.c_void_p(self.ptr))
            self.ptr = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def host_empty(shape, dtype) -> np.ndarray:
    """A zero-filled numpy array in ``ipg_host_alloc`` memory, for fast host <-> device copies."""
    dtype = np.dtype(dtype)
    shape = (int(shape),) if np.isscalar(shape) else tuple(int(s) for s in shape)
    count = int(np.prod(shape, dtype=np.int64))
    if count == 0:
        return np.zeros(shape, dtype=dtype)
    raw = np.asarray(HostBuffer(count * dtype.itemsize))
    return raw.view(dtype).reshape(shape)


__all__ += ["HostBuffer", "host_empty"]
