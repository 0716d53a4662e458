"""Seeded synthetic graph inputs shared by the CPU oracle and the GPU library.

The C code in ``graphgen.c`` produces edge lists and CSR arrays from a seed;
it contains no connectivity arithmetic.  This wrapper compiles it on first use
(``build()``) and exposes numpy-returning helpers.

Workload shapes stand in for the graphs of the paper's evaluation (Section 4,
Table 2), which are public datasets and are not used here:

* ``er``          Erdos-Renyi G(n, m) multigraph (self-loops, duplicates kept)
* ``rmat``        RMAT / Graph500 Kronecker edges, optional random relabelling
* ``grid_paths``  2D grid with random edge removal plus long permuted paths
* ``batched``     thousands of small ER / RMAT graphs with local ids
* ``ba``          Barabasi-Albert preferential attachment (streaming inputs)
* ``csr``         symmetric CSR with sorted rows built from a COO list
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

# Graph500 / paper RMAT parameters (a, b, c); d = 1 - a - b - c.
GRAPH500 = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so next to it (gcc, OpenMP).  No
    fused multiply-add contraction: the batched sizes' floating-point steps
    round the same way on every machine (aarch64 gcc contracts by default)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                                                         os.path.getmtime(__file__)):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32, u64, i32, dbl, vp = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_void_p)
            sig = {
                "gg_splitmix64_at": (u64, [u64, u64]),
                "gg_stream_base": (u64, [u64, u64]),
                "gg_hash_fill": (None, [u64, u64, u64, u64, vp]),
                "gg_permutation": (None, [u32, u64, u64, vp]),
                "gg_er": (None, [u32, u64, u64, vp]),
                "gg_rmat": (None, [i32, u64, u32, u32, u32, u64, vp, vp]),
                "gg_rmat_range": (None, [i32, u64, u64, u32, u32, u32, u64, vp, vp]),
                "gg_pairs_range": (None, [u32, u64, u64, u64, vp]),
                "gg_ba": (None, [u32, u32, u64, vp]),
                "gg_shuffle_edges": (None, [u64, u64, u64, vp]),
                "gg_grid_paths": (u64, [u32, u32, u32, u32, u64, vp]),
                "gg_batched_sizes": (None, [u32, u32, u32, dbl, dbl, u64, vp, vp]),
                "gg_batched_fill": (None, [u32, vp, vp, u32, u32, u32, u64, vp]),
                "gg_coo_to_csr": (i32, [u32, u64, vp, vp, vp]),
                "gg_num_threads": (i32, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _thresholds(abc):
    a, b, c = abc
    ta = int(round(a * 2**32))
    tab = int(round((a + b) * 2**32))
    tabc = int(round((a + b + c) * 2**32))
    return ta, tab, min(tabc, 2**32 - 1)


def splitmix64_at(base: int, i: int) -> int:
    return int(_load().gg_splitmix64_at(base, i))


def stream_base(seed: int, stream: int) -> int:
    return int(_load().gg_stream_base(seed, stream))


def hash_fill(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().gg_hash_fill(seed, stream, start, count, _ptr(out))
    return out


def permutation(n: int, seed: int, stream: int = 6) -> np.ndarray:
    out = np.empty(max(n, 1), dtype=np.uint32)[:n]
    _load().gg_permutation(n, seed, stream, _ptr(out))
    return out


def out_edges(m: int, out=None) -> np.ndarray:
    if out is not None:
        assert out.dtype == np.uint32 and out.shape == (m, 2) and out.flags.c_contiguous
        return out
    return np.empty((m, 2), dtype=np.uint32)


def er(n: int, m: int, seed: int, out=None) -> np.ndarray:
    """(m, 2) uint32 edges of an Erdos-Renyi multigraph on n vertices."""
    e = out_edges(m, out)
    if m:
        _load().gg_er(n, m, seed, _ptr(e))
    return e


def rmat(scale: int, m: int, seed: int, abc=GRAPH500, permute: bool = True, out=None) -> np.ndarray:
    """(m, 2) uint32 RMAT edges on 2**scale vertices; ids randomly permuted if asked."""
    e = out_edges(m, out)
    ta, tab, tabc = _thresholds(abc)
    perm = permutation(1 << scale, seed, 6) if permute else None
    if m:
        _load().gg_rmat(scale, m, ta, tab, tabc, seed, _ptr(perm), _ptr(e))
    return e


def rmat_range(scale: int, start: int, count: int, seed: int, perm=None, abc=GRAPH500, out=None):
    """Edges [start, start+count) of the RMAT stream of ``rmat`` (same seed)."""
    e = out_edges(count, out)
    ta, tab, tabc = _thresholds(abc)
    if count:
        _load().gg_rmat_range(scale, start, count, ta, tab, tabc, seed, _ptr(perm), _ptr(e))
    return e


def ba(n: int, d: int, seed: int, out=None) -> np.ndarray:
    """Barabasi-Albert graph: vertex v attaches d edges (v, w), w <= v chosen
    with probability proportional to degree (Batagelj-Brandes endpoint copying)."""
    e = out_edges(n * d, out)
    if n and d:
        _load().gg_ba(n, d, seed, _ptr(e))
    return e


def pairs_range(n: int, start: int, count: int, seed: int, out=None) -> np.ndarray:
    """Uniform random vertex pairs (queries) [start, start+count) of a seeded stream."""
    e = out_edges(count, out)
    if count:
        _load().gg_pairs_range(n, start, count, seed, _ptr(e))
    return e


def grid_paths(side: int, remove_p: float, npaths: int, plen: int, seed: int):
    """2D grid (side x side, edges removed with prob. remove_p) + npaths permuted paths.

    Returns (n, edges) with n = side*side + npaths*plen.
    """
    lib = _load()
    thr = int(round(remove_p * 2**32))
    m = int(lib.gg_grid_paths(side, thr, npaths, plen, seed, None))
    e = np.empty((m, 2), dtype=np.uint32)
    m2 = int(lib.gg_grid_paths(side, thr, npaths, plen, seed, _ptr(e)))
    assert m2 == m
    return side * side + npaths * plen, e


def path_permutation(npaths: int, plen: int, seed: int) -> np.ndarray:
    """The permutation grid_paths uses to lay out its paths (stream 4)."""
    return permutation(npaths * plen, seed, 4)


def batched(G: int, seed: int, nmin: int = 256, nmax: int = 65536, dmin: float = 4.0,
            dmax: float = 32.0, abc=GRAPH500):
    """G independent graphs with local ids.

    Returns (vtx_off[G+1] u64, edge_off[G+1] u64, edges (sum m_i, 2) u32).
    """
    lib = _load()
    vo = np.empty(G + 1, dtype=np.uint64)
    eo = np.empty(G + 1, dtype=np.uint64)
    lib.gg_batched_sizes(G, nmin, nmax, dmin, dmax, seed, _ptr(vo), _ptr(eo))
    e = np.empty((int(eo[-1]), 2), dtype=np.uint32)
    ta, tab, tabc = _thresholds(abc)
    lib.gg_batched_fill(G, _ptr(vo), _ptr(eo), ta, tab, tabc, seed, _ptr(e))
    return vo, eo, e


def csr(n: int, edges: np.ndarray):
    """Symmetric CSR (offsets u64[n+1], cols u32[2m]) with sorted rows."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    m = edges.shape[0]
    off = np.empty(n + 1, dtype=np.uint64)
    cols = np.empty(max(2 * m, 1), dtype=np.uint32)[: 2 * m]
    rc = _load().gg_coo_to_csr(n, m, _ptr(edges), _ptr(off), _ptr(cols))
    if rc != 0:
        raise ValueError(f"gg_coo_to_csr failed ({rc}): endpoint >= n or no memory")
    return off, cols


def num_threads() -> int:
    return int(_load().gg_num_threads())
