"""CPU baseline in the paper's final design (OpenMP on all host cores): PageRank and
Hashmin pulling from in-neighbours, SSSP pushing from the active list into
compare-and-swap mailboxes, dynamic schedule with chunks of 256.

A measured comparison point for the GPU library, beside the single-threaded oracle;
correctness is the oracle's job (the tests check this baseline against it).  Shares no
code with the library or the oracle.  Built on first use with gcc -fopenmp.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pregel_omp.c")
_SO = os.path.join(_HERE, "libpregel_omp.so")
_lib_handle = None


class BaselineError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
        pu32, pu64, pd = ctypes.POINTER(u32), ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)
        lib.pomp_pagerank.argtypes = [u32, vp, vp, u32, vp, pu64, pd, pd]
        lib.pomp_pagerank.restype = i32
        lib.pomp_sssp.argtypes = [u32, vp, vp, vp, u32, vp, pu32, pu64, pd]
        lib.pomp_sssp.restype = i32
        lib.pomp_hashmin.argtypes = [u32, vp, vp, vp, pu32, pu64, pd]
        lib.pomp_hashmin.restype = i32
        lib.pomp_threads.argtypes = []
        lib.pomp_threads.restype = i32
        _lib_handle = lib
    return _lib_handle


@dataclass
class Run:
    values: np.ndarray
    supersteps: int
    messages: int
    seconds: float          # the supersteps
    load_seconds: float = 0.0  # in-edge lists (pull programs)


def threads() -> int:
    return int(_lib().pomp_threads())


def _csr(n, offsets, cols, weights=None):
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    cols = np.ascontiguousarray(cols, dtype=np.uint32)
    if offsets.shape != (n + 1,):
        raise ValueError("offsets must have n+1 entries")
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.uint32)
    return offsets, cols, w


def _p(a: Optional[np.ndarray]):
    return None if a is None or a.size == 0 else a.ctypes.data


def pagerank(n: int, offsets, cols, updates: int = 10) -> Run:
    offsets, cols, _ = _csr(n, offsets, cols)
    rank = np.empty(max(n, 1), dtype=np.float32)
    msgs, sec, load = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
    rc = _lib().pomp_pagerank(n, _p(offsets), _p(cols), updates, rank.ctypes.data, ctypes.byref(msgs),
                              ctypes.byref(sec), ctypes.byref(load))
    if rc:
        raise BaselineError(f"pomp_pagerank failed with code {rc}")
    return Run(rank[:n], updates + 1, int(msgs.value), float(sec.value), float(load.value))


def sssp(n: int, offsets, cols, weights, source: int) -> Run:
    offsets, cols, w = _csr(n, offsets, cols, weights)
    dist = np.empty(max(n, 1), dtype=np.uint32)
    ss, msgs, sec = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_double()
    rc = _lib().pomp_sssp(n, _p(offsets), _p(cols), _p(w), source, dist.ctypes.data, ctypes.byref(ss),
                          ctypes.byref(msgs), ctypes.byref(sec))
    if rc:
        raise BaselineError(f"pomp_sssp failed with code {rc}")
    return Run(dist[:n], int(ss.value), int(msgs.value), float(sec.value))


def hashmin(n: int, offsets, cols) -> Run:
    offsets, cols, _ = _csr(n, offsets, cols)
    label = np.empty(max(n, 1), dtype=np.uint32)
    ss, msgs, sec = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_double()
    rc = _lib().pomp_hashmin(n, _p(offsets), _p(cols), label.ctypes.data, ctypes.byref(ss), ctypes.byref(msgs),
                             ctypes.byref(sec))
    if rc:
        raise BaselineError(f"pomp_hashmin failed with code {rc}")
    return Run(label[:n], int(ss.value), int(msgs.value), float(sec.value))
