"""CPU oracle for connectivity (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may import this package.  The GPU library never does, and this
package never imports the GPU library: the two share no code.  The seeded
input generators (``graphgen``) are the only module both sides use.

``oracle.c`` holds the sequential definitions (union-find O1, BFS O2, the
spanning-forest checker, the incremental replay); ``method_ref`` restates the
paper's per-step rules in plain Python for small inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SF_CODES = {
    0: "valid",
    1: "edge id out of range",
    2: "duplicate edge id",
    3: "self-loop in forest",
    4: "cycle in forest",
    5: "edge count != n - components",
    6: "forest partition differs from the components",
}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, single-threaded)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32, u64, i32, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
            sig = {
                "oracle_cc_uf": (i32, [u32, u64, vp, vp]),
                "oracle_cc_bfs": (i32, [u32, u64, vp, vp]),
                "oracle_sf_check": (i32, [u32, u64, vp, vp, u64, vp]),
                "oracle_sf_check_arcs": (i32, [u32, vp, vp, vp, u64, vp]),
                "oracle_kruskal_forest": (u64, [u32, u64, vp, vp]),
                "oracle_inc_new": (vp, [u32]),
                "oracle_inc_insert": (i32, [vp, u64, vp]),
                "oracle_inc_query": (i32, [vp, u64, vp, vp]),
                "oracle_inc_labels": (None, [vp, vp]),
                "oracle_inc_free": (None, [vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _edges(edges) -> np.ndarray:
    e = np.ascontiguousarray(edges, dtype=np.uint32).reshape(-1, 2)
    return e


def cc_uf(n: int, edges) -> np.ndarray:
    """O1: canonical (min-id) component labels by sequential union-find."""
    e = _edges(edges)
    out = np.empty(max(n, 1), dtype=np.uint32)[:n]
    rc = _load().oracle_cc_uf(n, e.shape[0], _p(e), _p(out))
    if rc:
        raise ValueError("endpoint >= n")
    return out


def cc_bfs(n: int, edges) -> np.ndarray:
    """O2: canonical (min-id) component labels by BFS in increasing id order."""
    e = _edges(edges)
    out = np.empty(max(n, 1), dtype=np.uint32)[:n]
    rc = _load().oracle_cc_bfs(n, e.shape[0], _p(e), _p(out))
    if rc:
        raise ValueError("endpoint >= n")
    return out


def sf_check(n: int, edges, ids, ref_labels) -> int:
    """Check a spanning forest given as COO edge indices; 0 = valid (see SF_CODES)."""
    e = _edges(edges)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    ref = np.ascontiguousarray(ref_labels, dtype=np.uint32)
    return int(_load().oracle_sf_check(n, e.shape[0], _p(e), _p(ids), ids.shape[0], _p(ref)))


def sf_check_arcs(n: int, offsets, cols, ids, ref_labels) -> int:
    """Check a spanning forest given as CSR arc positions; 0 = valid."""
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    cols = np.ascontiguousarray(cols, dtype=np.uint32)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    ref = np.ascontiguousarray(ref_labels, dtype=np.uint32)
    return int(_load().oracle_sf_check_arcs(n, _p(off), _p(cols), _p(ids), ids.shape[0], _p(ref)))


def kruskal_forest(n: int, edges) -> np.ndarray:
    e = _edges(edges)
    ids = np.empty(max(n, 1), dtype=np.uint64)
    c = int(_load().oracle_kruskal_forest(n, e.shape[0], _p(e), _p(ids)))
    return ids[:c]


class Incremental:
    """Sequential replay of an insert / query stream (Section 3.5 semantics)."""

    def __init__(self, n: int):
        self.n = n
        self._h = _load().oracle_inc_new(n)

    def insert(self, edges) -> None:
        e = _edges(edges)
        if _load().oracle_inc_insert(self._h, e.shape[0], _p(e)):
            raise ValueError("endpoint >= n")

    def query(self, pairs) -> np.ndarray:
        e = _edges(pairs)
        out = np.empty(max(e.shape[0], 1), dtype=np.uint8)[: e.shape[0]]
        if _load().oracle_inc_query(self._h, e.shape[0], _p(e), _p(out)):
            raise ValueError("endpoint >= n")
        return out

    def labels(self) -> np.ndarray:
        out = np.empty(max(self.n, 1), dtype=np.uint32)[: self.n]
        _load().oracle_inc_labels(self._h, _p(out))
        return out

    def close(self) -> None:
        if self._h:
            _load().oracle_inc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batched_cc(vtx_off, edge_off, edges) -> np.ndarray:
    """O1 applied to every graph of a batch (local ids in, local min ids out)."""
    vo = np.asarray(vtx_off, dtype=np.uint64)
    eo = np.asarray(edge_off, dtype=np.uint64)
    e = _edges(edges)
    out = np.empty(int(vo[-1]), dtype=np.uint32)
    for g in range(len(vo) - 1):
        n = int(vo[g + 1] - vo[g])
        out[int(vo[g]):int(vo[g + 1])] = cc_uf(n, e[int(eo[g]):int(eo[g + 1])])
    return out
