"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds none of the method's arithmetic: it only produces graphs as a
CSR of out-links (``row_ptr`` int32[n+1], ``col_idx`` int32[L], each row sorted
ascending) and personalization seed sets.  The C source ``graphgen.c`` is
compiled with gcc on first use (and by ``__graft_entry__.build()``).

Families (synthetic stand-ins for the power-law graphs of the paper's
Section 4.1 and for the public web graphs of Section 4.3):

* :func:`uniform_graph`  -- out-degree U{0..dmax}, uniform distinct targets.
* :func:`zipf_graph`     -- exact dangling fraction, Zipf out-degrees clipped at
  ``kmax``, targets drawn proportional to rank^-beta over permuted ids.
* :func:`rmat_graph`     -- R-MAT with quadrant probabilities (a, b, c, d).
* :func:`seed_set` / :func:`seed_sets` -- personalization seed nodes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``graphgen.c`` into ``libgraphgen.so`` next to it."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i32p = ctypes.POINTER(ctypes.c_int32)
    u64 = ctypes.c_uint64
    lib.gg_uniform_degrees.argtypes = [ctypes.c_int32, ctypes.c_int32, u64, i32p]
    lib.gg_uniform_degrees.restype = ctypes.c_int64
    lib.gg_uniform_fill.argtypes = [ctypes.c_int32, u64, i32p, i32p]
    lib.gg_uniform_fill.restype = None
    lib.gg_zipf_degrees.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_double, u64, i32p]
    lib.gg_zipf_degrees.restype = ctypes.c_int64
    lib.gg_zipf_fill.argtypes = [ctypes.c_int32, ctypes.c_double, u64, i32p, i32p]
    lib.gg_zipf_fill.restype = ctypes.c_int
    lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            u64, ctypes.c_int, i32p, i32p]
    lib.gg_rmat.restype = ctypes.c_int64
    lib.gg_seed_set.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, u64, ctypes.c_int64, i32p]
    lib.gg_seed_set.restype = ctypes.c_int32
    lib.gg_unit.argtypes = [u64, u64, u64]
    lib.gg_unit.restype = ctypes.c_double
    lib.gg_modify.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_double, ctypes.c_int64, u64, i32p, i32p,
                              ctypes.c_int64]
    lib.gg_modify.restype = ctypes.c_int64
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


@dataclass
class Graph:
    """A directed graph as a CSR of out-links: row i lists the children of node i."""

    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col_idx: np.ndarray  # int32[L]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def outdeg(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


def uniform_graph(n: int, dmax: int = 20, seed: int = 1) -> Graph:
    """Out-degree uniform in {0..dmax}; targets uniform over the other nodes, distinct."""
    lib = _load()
    row_ptr = np.empty(n + 1, dtype=np.int32)
    tot = lib.gg_uniform_degrees(n, dmax, seed, _p(row_ptr))
    if tot < 0:
        raise ValueError("uniform_graph: bad size")
    col_idx = np.empty(max(tot, 1), dtype=np.int32)
    lib.gg_uniform_fill(n, seed, _p(row_ptr), _p(col_idx))
    return Graph(n, row_ptr, col_idx[:tot], f"uniform(n={n},dmax={dmax},seed={seed})")


def zipf_graph(n: int, alpha: float = 2.1, kmax: int = 50000, dangling_frac: float = 0.12,
               target_exp: float = 0.9, seed: int = 1) -> Graph:
    """Exact floor(frac*n) dangling nodes; other out-degrees Zipf(alpha) clipped at kmax;
    targets proportional to rank^-target_exp over a seeded permutation of ids."""
    lib = _load()
    row_ptr = np.empty(n + 1, dtype=np.int32)
    tot = lib.gg_zipf_degrees(n, alpha, kmax, dangling_frac, seed, _p(row_ptr))
    if tot < 0:
        raise ValueError("zipf_graph: bad parameters or more than 2^31-1 edges")
    col_idx = np.empty(max(tot, 1), dtype=np.int32)
    if lib.gg_zipf_fill(n, target_exp, seed, _p(row_ptr), _p(col_idx)) != 0:
        raise MemoryError("zipf_graph: allocation failed")
    return Graph(n, row_ptr, col_idx[:tot],
                 f"zipf(n={n},alpha={alpha},kmax={kmax},dangling={dangling_frac},beta={target_exp},seed={seed})")


def rmat_graph(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = 1, dedup: bool = True) -> Graph:
    """R-MAT with 2^scale nodes and edge_factor*2^scale draws; duplicates removed if dedup."""
    lib = _load()
    n = 1 << scale
    row_ptr = np.empty(n + 1, dtype=np.int32)
    col_idx = np.empty(edge_factor * n, dtype=np.int32)
    tot = lib.gg_rmat(scale, edge_factor, a, b, c, seed, 1 if dedup else 0, _p(row_ptr), _p(col_idx))
    if tot < 0:
        raise ValueError("rmat_graph: bad parameters")
    return Graph(n, row_ptr, col_idx[:tot].copy(),
                 f"rmat(scale={scale},ef={edge_factor},abc=({a},{b},{c}),seed={seed},dedup={dedup})")


def modify(g: Graph, drop: float, extra: int, seed: int) -> Graph:
    """An edited copy: each edge dropped with probability `drop`, `extra` uniform random edges added."""
    lib = _load()
    cap = len(g.col_idx) + int(extra)
    row_ptr = np.empty(g.n + 1, dtype=np.int32)
    col_idx = np.empty(max(cap, 1), dtype=np.int32)
    tot = lib.gg_modify(g.n, _p(np.ascontiguousarray(g.row_ptr, np.int32)),
                        _p(np.ascontiguousarray(g.col_idx if len(g.col_idx) else np.zeros(1, np.int32), np.int32)),
                        float(drop), int(extra), seed, _p(row_ptr), _p(col_idx), cap)
    if tot < 0:
        raise ValueError("modify: output capacity exceeded")
    return Graph(g.n, row_ptr, col_idx[:tot].copy(), f"modify({g.name},drop={drop},extra={extra},seed={seed})")


def seed_set(n: int, smin: int, smax: int, seed: int, q: int) -> np.ndarray:
    """Seed nodes of query q: size uniform in {smin..smax}, distinct, uniform over [0, n)."""
    lib = _load()
    out = np.empty(max(smax, 1), dtype=np.int32)
    sz = lib.gg_seed_set(n, smin, smax, seed, q, _p(out))
    if sz < 0:
        raise ValueError("seed_set: bad parameters")
    return out[:sz].copy()


def seed_sets(n: int, k: int, smin: int, smax: int, seed: int, first: int = 0) -> list:
    return [seed_set(n, smin, smax, seed, first + q) for q in range(k)]


def uniform_v(n: int) -> np.ndarray:
    """The uniform personalization vector V = 1/N."""
    return np.full(n, 1.0 / n, dtype=np.float64)


def unit_draw(seed: int, stream: int, ctr: int) -> float:
    return _load().gg_unit(seed, stream, ctr)
