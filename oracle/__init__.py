"""ORACLE — test infrastructure only.

Python access to the plain single-threaded CPU Pregel implementation in
``oracle/ipg_oracle.c`` (PageRank in float64, Hashmin connected components, SSSP,
the shortest-path tree and shortest-path counting with wider messages, and the
mailbox combination step alone), written from the paper's description of the
vertex-centric model (Sec. I) and of the mailbox with its "has a message" flag
and user-defined combine function (Sec. III, Fig. 1).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may import this package.  The library under
``paper_2010_01542_gb300/`` never does; the two share no code.

Every function here is pinned by ``tests/test_oracle_pins.py`` against closed
forms, scipy routines, a dense linear solve and counting identities.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ipg_oracle.c")
_SO = os.path.join(_HERE, "libipg_oracle.so")
_lib_handle = None

INF = 0xFFFFFFFF


class OracleError(RuntimeError):
    pass


class _Stats(ctypes.Structure):
    _fields_ = [("superstep", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("active", ctypes.c_uint64),
                ("senders", ctypes.c_uint64), ("messages_sent", ctypes.c_uint64), ("receivers", ctypes.c_uint64)]


@dataclass
class SuperstepStats:
    superstep: int
    active: int
    senders: int
    messages_sent: int
    receivers: int


@dataclass
class Result:
    values: np.ndarray
    supersteps: int
    stats: List[SuperstepStats]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, gcc -O2, no arch-specific flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        path = os.environ.get("IPG_ORACLE_LIB")  # another build of the oracle (the mutation tests' mutants)
        if not path:
            build()
            path = _SO
        lib = ctypes.CDLL(path)
        vp, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
        lib.orc_hashmin.argtypes = [u32, vp, vp, vp, vp, u32, u32, ctypes.POINTER(u32)]
        lib.orc_hashmin.restype = i32
        lib.orc_sssp.argtypes = [u32, vp, vp, vp, u32, vp, vp, u32, u32, ctypes.POINTER(u32)]
        lib.orc_sssp.restype = i32
        lib.orc_pagerank.argtypes = [u32, vp, vp, u32, vp, vp, u32, ctypes.POINTER(u32)]
        lib.orc_pagerank.restype = i32
        lib.orc_combine.argtypes = [i32, u32, ctypes.c_uint64, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
        lib.orc_combine.restype = i32
        lib.orc_sssp_tree.argtypes = [u32, vp, vp, vp, u32, vp, vp, vp, u32, u32, ctypes.POINTER(u32)]
        lib.orc_sssp_tree.restype = i32
        lib.orc_bfs_paths.argtypes = [u32, vp, vp, u32, vp, vp, vp, u32, u32, ctypes.POINTER(u32)]
        lib.orc_bfs_paths.restype = i32
        _lib_handle = lib
    return _lib_handle


def _ptr(a: Optional[np.ndarray]):
    return None if a is None or a.size == 0 else a.ctypes.data


def _prep(n, offsets, cols, weights=None):
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    cols = np.ascontiguousarray(cols, dtype=np.uint32)
    if offsets.shape != (n + 1,):
        raise ValueError("offsets must have n+1 entries")
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.uint32)
    return offsets, cols, w


def _stats(buf, k) -> List[SuperstepStats]:
    return [SuperstepStats(int(buf[i].superstep), int(buf[i].active), int(buf[i].senders),
                           int(buf[i].messages_sent), int(buf[i].receivers)) for i in range(k)]


_CAP = 1 << 16


def hashmin(n: int, offsets, cols, max_supersteps: int = 0) -> Result:
    offsets, cols, _ = _prep(n, offsets, cols)
    label = np.empty(max(n, 1), dtype=np.uint32)
    st = (_Stats * _CAP)()
    ss = ctypes.c_uint32()
    rc = _lib().orc_hashmin(n, _ptr(offsets), _ptr(cols), label.ctypes.data, st, _CAP, max_supersteps,
                            ctypes.byref(ss))
    if rc:
        raise OracleError(f"orc_hashmin failed with code {rc}")
    return Result(label[:n], int(ss.value), _stats(st, min(ss.value, _CAP)))


def sssp(n: int, offsets, cols, weights, source: int, max_supersteps: int = 0) -> Result:
    offsets, cols, w = _prep(n, offsets, cols, weights)
    dist = np.empty(max(n, 1), dtype=np.uint32)
    st = (_Stats * _CAP)()
    ss = ctypes.c_uint32()
    rc = _lib().orc_sssp(n, _ptr(offsets), _ptr(cols), _ptr(w), source, dist.ctypes.data, st, _CAP,
                         max_supersteps, ctypes.byref(ss))
    if rc:
        raise OracleError(f"orc_sssp failed with code {rc}")
    return Result(dist[:n], int(ss.value), _stats(st, min(ss.value, _CAP)))


def pagerank(n: int, offsets, cols, updates: int = 10) -> Result:
    offsets, cols, _ = _prep(n, offsets, cols)
    rank = np.empty(max(n, 1), dtype=np.float64)
    st = (_Stats * _CAP)()
    ss = ctypes.c_uint32()
    rc = _lib().orc_pagerank(n, _ptr(offsets), _ptr(cols), updates, rank.ctypes.data, st, _CAP, ctypes.byref(ss))
    if rc:
        raise OracleError(f"orc_pagerank failed with code {rc}")
    return Result(rank[:n], int(ss.value), _stats(st, min(ss.value, _CAP)))


# combine kinds of orc_combine (same numbering as the C ABI's ipg_combine_kind)
COMBINE_XOR_U32 = 0
COMBINE_MIN_U64 = 1
COMBINE_SUM_U64 = 2
COMBINE_MINCOUNT_U128 = 3
_KIND_DTYPE = {COMBINE_XOR_U32: (np.uint32, 1), COMBINE_MIN_U64: (np.uint64, 1), COMBINE_SUM_U64: (np.uint64, 1),
               COMBINE_MINCOUNT_U128: (np.uint64, 2)}


@dataclass
class CombineResult:
    has: np.ndarray       # bool[n]: the vertex received at least one message
    mail: np.ndarray      # combined message per vertex (meaningful where has is True)
    receivers: int


def combine(kind: int, n: int, dst, msgs) -> CombineResult:
    """Deliver messages msgs[i] to dst[i] into n empty mailboxes (Sec. III).  msgs is a
    u32[k] (XOR_U32), u64[k] (MIN_U64, SUM_U64) or u64[k, 2] = (key, count) (MINCOUNT_U128)."""
    dt, width = _KIND_DTYPE[kind]
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    msgs = np.ascontiguousarray(msgs, dtype=dt)
    k = dst.shape[0]
    if msgs.shape != ((k,) if width == 1 else (k, 2)):
        raise ValueError("message array has the wrong shape for this kind")
    has = np.zeros(max(n, 1), dtype=np.uint8)
    mail = np.zeros((max(n, 1),) if width == 1 else (max(n, 1), 2), dtype=dt)
    r = ctypes.c_uint64()
    rc = _lib().orc_combine(kind, n, k, _ptr(dst), _ptr(msgs), has.ctypes.data, mail.ctypes.data, ctypes.byref(r))
    if rc:
        raise OracleError(f"orc_combine failed with code {rc}")
    return CombineResult(has[:n].astype(bool), mail[:n], int(r.value))


@dataclass
class TreeResult:
    dist: np.ndarray
    parent: np.ndarray
    supersteps: int
    stats: List[SuperstepStats]


def sssp_tree(n: int, offsets, cols, weights, source: int, max_supersteps: int = 0) -> TreeResult:
    offsets, cols, w = _prep(n, offsets, cols, weights)
    dist = np.empty(max(n, 1), dtype=np.uint32)
    parent = np.empty(max(n, 1), dtype=np.uint32)
    st = (_Stats * _CAP)()
    ss = ctypes.c_uint32()
    rc = _lib().orc_sssp_tree(n, _ptr(offsets), _ptr(cols), _ptr(w), source, dist.ctypes.data, parent.ctypes.data,
                              st, _CAP, max_supersteps, ctypes.byref(ss))
    if rc:
        raise OracleError(f"orc_sssp_tree failed with code {rc}")
    return TreeResult(dist[:n], parent[:n], int(ss.value), _stats(st, min(ss.value, _CAP)))


@dataclass
class PathsResult:
    level: np.ndarray
    paths: np.ndarray
    supersteps: int
    stats: List[SuperstepStats]


def bfs_paths(n: int, offsets, cols, source: int, max_supersteps: int = 0) -> PathsResult:
    offsets, cols, _ = _prep(n, offsets, cols)
    level = np.empty(max(n, 1), dtype=np.uint32)
    paths = np.empty(max(n, 1), dtype=np.uint64)
    st = (_Stats * _CAP)()
    ss = ctypes.c_uint32()
    rc = _lib().orc_bfs_paths(n, _ptr(offsets), _ptr(cols), source, level.ctypes.data, paths.ctypes.data, st, _CAP,
                              max_supersteps, ctypes.byref(ss))
    if rc:
        raise OracleError(f"orc_bfs_paths failed with code {rc}")
    return PathsResult(level[:n], paths[:n], int(ss.value), _stats(st, min(ss.value, _CAP)))
