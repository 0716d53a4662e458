"""Multicore CPU baseline: the two-phase connectivity method on the host
cores (OpenMP threads, lock-free union-find), the local analogue of the
paper's GPU-versus-multicore comparison (Section 4.8).

A measured baseline for ``bench.py``, not a parity reference (the oracle is
that); the CPU tests check its labels against the oracle.  Nothing in the GPU
library imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mt_cc.c")
_LIB = os.path.join(_HERE, "libmtcc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile mt_cc.c into libmtcc.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.mt_cc_csr.restype = ctypes.c_int
            lib.mt_cc_csr.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
            lib.mt_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().mt_max_threads())


def cc_csr(n: int, off: np.ndarray, cols: np.ndarray, k: int = 2, threads: int = 0,
           seed: int = 0x6C0A0001, out: np.ndarray | None = None) -> np.ndarray:
    """Canonical labels (smallest id per component) of a symmetric CSR graph."""
    off = np.ascontiguousarray(off, dtype=np.uint64)
    cols = np.ascontiguousarray(cols, dtype=np.uint32)
    assert off.shape == (n + 1,)
    lab = out if out is not None else np.empty(max(n, 1), np.uint32)[:n]
    rc = _load().mt_cc_csr(n, off.ctypes.data, cols.ctypes.data if cols.size else None, lab.ctypes.data,
                           k, threads, seed)
    if rc == 1:
        raise ValueError("column entry out of range")
    if rc != 0:
        raise MemoryError("mt_cc_csr: allocation failed")
    return lab
