"""Seeded synthetic graph inputs shared by the tests, the benchmark and the oracle side.

This module holds no Pregel arithmetic.  It produces the CSR graphs that both the
CUDA path and the CPU oracle take as input:

* ``rmat``: R-MAT power-law graphs (Chakrabarti et al. 2004) from a counter-based
  splitmix64 stream; they stand in for the SNAP social graphs of the paper's
  Table I (Sec. VI-B), which are not available here.  The recipe is in
  ``gen/rmat.c``.
* ``csr_from_edges``: exact CSR from a hand-written edge list, keeping self-loops and
  multi-edges unless asked otherwise (adversarial test graphs).
* ``edge_weights``: per-edge weights in [1, wmax] from the edge's endpoints.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmat.c")
_SO = os.path.join(_HERE, "libipg_gen.so")
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile the generator's C code into ``gen/libipg_gen.so`` (gcc, no arch flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_SO)
        u32, u64, i32, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        vp = ctypes.c_void_p
        lib.gen_rmat_plan.argtypes = [u32, u32, dbl, dbl, dbl, u64, i32, i32,
                                      ctypes.POINTER(vp), ctypes.POINTER(u32), ctypes.POINTER(u64)]
        lib.gen_rmat_plan.restype = i32
        lib.gen_plan_emit.argtypes = [vp, vp, vp]
        lib.gen_plan_emit.restype = i32
        lib.gen_plan_free.argtypes = [vp]
        lib.gen_plan_free.restype = None
        lib.gen_weights.argtypes = [u32, vp, vp, u64, u32, i32, i32, vp]
        lib.gen_weights.restype = i32
        lib.gen_splitmix64.argtypes = [u64]
        lib.gen_splitmix64.restype = u64
        _lib_handle = lib
    return _lib_handle


@dataclass
class CSR:
    """A graph in compressed sparse row form (out-edges of vertex u are
    ``cols[offsets[u]:offsets[u+1]]``)."""

    n: int
    offsets: np.ndarray  # uint64[n+1]
    cols: np.ndarray  # uint32[m]
    weights: Optional[np.ndarray] = None  # uint32[m] or None
    directed: bool = True

    @property
    def m(self) -> int:
        return int(self.offsets[-1]) if self.n >= 0 else 0

    def out_degree(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))


def splitmix64(x: int) -> int:
    return int(_lib().gen_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def default_weight_seed(seed: int) -> int:
    """Weight stream seed derived from the graph seed (documented constant)."""
    return (seed ^ 0x5EED_0F_0EED) & 0xFFFFFFFFFFFFFFFF


def _np_alloc(shape, dtype):
    return np.empty(shape, dtype=dtype)


def rmat(scale: int, edge_factor: int, seed: int = 1, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         undirected: bool = False, weighted: bool = False, weight_seed: Optional[int] = None, wmax: int = 255,
         nthreads: int = 0, alloc: Callable = _np_alloc) -> CSR:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale sampled edges, self-loops
    dropped, each row sorted and deduplicated (undirected: symmetrised before dedup).

    ``alloc(shape, dtype)`` provides the output arrays (e.g. views of pinned host memory).
    """
    lib = _lib()
    plan = ctypes.c_void_p()
    n = ctypes.c_uint32()
    m = ctypes.c_uint64()
    rc = lib.gen_rmat_plan(scale, edge_factor, a, b, c, seed & 0xFFFFFFFFFFFFFFFF, int(undirected), nthreads,
                           ctypes.byref(plan), ctypes.byref(n), ctypes.byref(m))
    if rc != 0:
        raise ValueError(f"gen_rmat_plan failed with code {rc}")
    try:
        offsets = alloc((n.value + 1,), np.uint64)
        cols = alloc((max(m.value, 0),), np.uint32)
        rc = lib.gen_plan_emit(plan, offsets.ctypes.data, cols.ctypes.data if m.value else None)
        if rc != 0:
            raise RuntimeError(f"gen_plan_emit failed with code {rc}")
    finally:
        lib.gen_plan_free(plan)
    g = CSR(n=n.value, offsets=offsets, cols=cols, weights=None, directed=not undirected)
    if weighted:
        ws = default_weight_seed(seed) if weight_seed is None else weight_seed
        g.weights = edge_weights(g.n, g.offsets, g.cols, ws, wmax=wmax, symmetric=undirected,
                                 nthreads=nthreads, out=alloc((g.m,), np.uint32))
    return g


def edge_weights(n: int, offsets: np.ndarray, cols: np.ndarray, weight_seed: int, wmax: int = 255,
                 symmetric: bool = False, nthreads: int = 0, out: Optional[np.ndarray] = None) -> np.ndarray:
    """Weights in [1, wmax] that depend only on (weight_seed, endpoints)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    cols = np.ascontiguousarray(cols, dtype=np.uint32)
    m = int(offsets[n])
    if out is None:
        out = np.empty(m, dtype=np.uint32)
    rc = _lib().gen_weights(n, offsets.ctypes.data, cols.ctypes.data if m else None,
                            weight_seed & 0xFFFFFFFFFFFFFFFF, wmax, int(symmetric), nthreads,
                            out.ctypes.data if m else None)
    if rc != 0:
        raise ValueError(f"gen_weights failed with code {rc}")
    return out


def csr_from_edges(n: int, src, dst, weights=None, undirected: bool = False, dedup: bool = False,
                   drop_self_loops: bool = False) -> CSR:
    """CSR from an explicit edge list.  Rows are sorted by destination (stable, so the
    relative order of parallel edges is kept).  By default self-loops and multi-edges
    are kept: each is one edge and carries one message."""
    src = np.asarray(src, dtype=np.int64).ravel()
    dst = np.asarray(dst, dtype=np.int64).ravel()
    w = None if weights is None else np.asarray(weights, dtype=np.int64).ravel()
    if src.shape != dst.shape or (w is not None and w.shape != src.shape):
        raise ValueError("edge arrays differ in length")
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("vertex id out of range")
    if drop_self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
        w = None if w is None else w[keep]
    if undirected:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
        w = None if w is None else np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    w = None if w is None else w[order]
    if dedup and src.size:
        keep = np.ones(src.size, dtype=bool)
        keep[1:] = (src[1:] != src[:-1]) | (dst[1:] != dst[:-1])
        src, dst = src[keep], dst[keep]
        w = None if w is None else w[keep]
    counts = np.bincount(src, minlength=n).astype(np.uint64) if src.size else np.zeros(n, dtype=np.uint64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=offsets[1:])
    return CSR(n=n, offsets=offsets, cols=dst.astype(np.uint32),
               weights=None if w is None else w.astype(np.uint32), directed=not undirected)


def max_out_degree_vertex(g: CSR) -> int:
    """Vertex with the largest out-degree, lowest id on ties."""
    if g.n == 0:
        raise ValueError("empty graph")
    return int(np.argmax(g.out_degree()))


def random_multigraph(n: int, m: int, seed: int, undirected: bool = False, weighted: bool = False,
                      wmax: int = 255, self_loops: bool = True) -> CSR:
    """Uniform random multigraph (numpy PCG64 stream): m edges drawn with
    replacement, so parallel edges and (unless disabled) self-loops occur."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, size=m) if n else np.zeros(0, dtype=np.int64)
    dst = rng.integers(0, n, size=m) if n else np.zeros(0, dtype=np.int64)
    if not self_loops and m:
        dst = np.where(dst == src, (dst + 1) % n, dst) if n > 1 else dst[:0]
        src = src[:dst.size]
    w = rng.integers(1, wmax + 1, size=src.size) if weighted else None
    return csr_from_edges(n, src, dst, w, undirected=undirected)


# ---------------------------------------------------------------------------------------
# GPU build of the same R-MAT graphs (gen/rmat_cuda.cu): bit-identical CSR, seconds
# instead of minutes for the billion-edge graphs.

_CUDA_SRC = os.path.join(_HERE, "rmat_cuda.cu")
_CUDA_SO = os.path.join(_HERE, "libipg_gen_cuda.so")
_cuda_handle = None


def build_cuda(force: bool = False) -> str:
    """Compile gen/rmat_cuda.cu for sm_103a (needs nvcc; no GPU needed to build)."""
    if force or not os.path.exists(_CUDA_SO) or os.path.getmtime(_CUDA_SO) < os.path.getmtime(_CUDA_SRC):
        nvcc = os.environ.get("NVCC") or "nvcc"
        tmp = _CUDA_SO + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                               "-Xcompiler", "-fPIC", "-shared", _CUDA_SRC, "-o", tmp])
        os.replace(tmp, _CUDA_SO)
    return _CUDA_SO


def _cuda_lib():
    global _cuda_handle
    if _cuda_handle is None:
        if not os.path.exists(_CUDA_SO):
            raise RuntimeError(f"{_CUDA_SO} is missing: build it with gen.build_cuda()")
        lib = ctypes.CDLL(_CUDA_SO)
        u32, u64, i32, dbl, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        lib.gen_rmat_cuda_plan.argtypes = [u32, u32, dbl, dbl, dbl, u64, i32, vp, ctypes.POINTER(vp),
                                           ctypes.POINTER(u32), ctypes.POINTER(u64)]
        lib.gen_rmat_cuda_plan.restype = i32
        lib.gen_rmat_cuda_emit.argtypes = [vp, vp, vp, vp, u64, u32, vp]
        lib.gen_rmat_cuda_emit.restype = i32
        lib.gen_rmat_cuda_free.argtypes = [vp]
        lib.gen_rmat_cuda_free.restype = None
        _cuda_handle = lib
    return _cuda_handle


@dataclass
class DeviceCSR:
    """CSR held in torch CUDA tensors (offsets as int64 bit patterns of uint64, columns
    and weights as int32 bit patterns of uint32)."""

    n: int
    m: int
    offsets: "object"
    cols: "object"
    weights: "object" = None
    directed: bool = True

    def to_host(self, pinned: bool = False, alloc=None) -> CSR:
        """Copy to host arrays: pageable, torch page-locked (``pinned``), or from ``alloc(shape, dtype)``."""
        import torch

        def cp(t, np_dtype):
            if t is None:
                return None
            if alloc is not None:
                h = alloc(tuple(t.shape), np_dtype)
                torch.from_numpy(h.view(np.dtype("i%d" % h.itemsize))).copy_(t)
                return h
            h = torch.empty(t.shape, dtype=t.dtype, pin_memory=pinned)
            h.copy_(t)
            return h.numpy().view(np_dtype)

        return CSR(n=self.n, offsets=cp(self.offsets, np.uint64), cols=cp(self.cols, np.uint32),
                   weights=cp(self.weights, np.uint32), directed=self.directed)


def rmat_device(scale: int, edge_factor: int, seed: int = 1, a: float = 0.57, b: float = 0.19, c: float = 0.19,
                undirected: bool = False, weighted: bool = False, weight_seed: Optional[int] = None,
                wmax: int = 255, device: int = 0) -> DeviceCSR:
    """Same graph as ``rmat(...)``, built on a CUDA device into torch tensors."""
    import torch

    lib = _cuda_lib()
    with torch.cuda.device(device):
        stream = torch.cuda.current_stream()
        sp = ctypes.c_void_p(int(stream.cuda_stream))
        plan, n, m = ctypes.c_void_p(), ctypes.c_uint32(), ctypes.c_uint64()
        torch.cuda.synchronize()
        rc = lib.gen_rmat_cuda_plan(scale, edge_factor, a, b, c, seed & 0xFFFFFFFFFFFFFFFF, int(undirected), sp,
                                    ctypes.byref(plan), ctypes.byref(n), ctypes.byref(m))
        if rc != 0:
            raise RuntimeError(f"gen_rmat_cuda_plan failed with code {rc}")
        try:
            offsets = torch.empty(n.value + 1, dtype=torch.int64, device="cuda")
            cols = torch.empty(max(m.value, 1), dtype=torch.int32, device="cuda")
            w = torch.empty(max(m.value, 1), dtype=torch.int32, device="cuda") if weighted else None
            ws = default_weight_seed(seed) if weight_seed is None else weight_seed
            rc = lib.gen_rmat_cuda_emit(plan, offsets.data_ptr(), cols.data_ptr(),
                                        w.data_ptr() if w is not None else None, ws & 0xFFFFFFFFFFFFFFFF, wmax, sp)
            if rc != 0:
                raise RuntimeError(f"gen_rmat_cuda_emit failed with code {rc}")
        finally:
            lib.gen_rmat_cuda_free(plan)
    return DeviceCSR(n=n.value, m=m.value, offsets=offsets, cols=cols[:m.value],
                     weights=None if w is None else w[:m.value], directed=not undirected)


# ---------------------------------------------------------------------------------------
# Workload recipes: the seeded choices (graph sizes, query sources) of the batched and
# served workloads, shared by bench.py and the tests that hold those workloads to the oracle.


def _splitmix_draws(count: int, seed: int):
    base = splitmix64(seed)
    return [splitmix64((base + i) & 0xFFFFFFFFFFFFFFFF) for i in range(count)]


def cc_batch_scales(count: int = 64, seed: int = 1):
    """Many-graph Hashmin: scale_i = 10 + splitmix64(splitmix64(seed) + i) % 11 (2^10 .. 2^20
    vertices), undirected, EF 16, graph seed i + 1."""
    return [10 + d % 11 for d in _splitmix_draws(count, seed)]


def serve_scales(count: int = 32, seed: int = 1):
    """Served graph set: scale_i = 12 + splitmix64(splitmix64(seed) + i) % 11 (2^12 .. 2^22
    vertices), undirected, weighted, EF 16, graph seed 101 + i."""
    return [12 + d % 11 for d in _splitmix_draws(count, seed)]


def batch_sources(n: int, k: int = 256, seed: int = 1) -> np.ndarray:
    """Many-source SSSP: k sources uniform on [0, n) from numpy's PCG64 stream of `seed`."""
    return np.random.default_rng(seed).integers(0, n, size=k).astype(np.uint32)
