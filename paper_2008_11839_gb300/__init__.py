"""GB300-native connected components and spanning forests (libgconn).

The compute path is the CUDA library ``libgconn.so`` (sources in ``csrc/``,
ABI in ``include/gconn.h``); this package only marshals arguments to it and
allocates output tensors with torch.  Build it with ``build()`` (nvcc,
sm_103a).  Functions named ``gconn_*`` mirror the C ABI one to one; ``cc``,
``cc_csr``, ``spanning_forest`` and ``Incremental`` are conveniences that
allocate the outputs.
"""
from __future__ import annotations

from ._binding import *  # noqa: F401,F403  (gconn_* wrappers, enums, errors)
from ._binding import (GconnError, GconnUnavailable, check, lib, make_variant, ptr,  # noqa: F401
                       stream_handle)


def build(force: bool = False) -> str:
    """Compile libgconn.so for sm_103a (in-tree)."""
    from ._build import build as _b
    return _b(force=force)


def _torch():
    import torch
    return torch


def cc(n: int, edges, variant=None, stream=None):
    """Canonical component labels (uint32 as int32 storage) of a COO edge list.

    ``edges`` is an (m, 2) int32/uint32-compatible tensor; labels are allocated
    on the same device.
    """
    torch = _torch()
    m = int(edges.shape[0]) if edges is not None else 0
    labels = torch.empty(n, dtype=torch.int32, device=edges.device)
    gconn_cc(n, m, edges, labels, variant, stream)  # noqa: F405
    return labels


def _off32(offsets) -> bool:
    """uint32 offsets: an int32 / uint32 tensor or array (else uint64)."""
    dt = str(getattr(offsets, "dtype", ""))
    return dt.endswith("int32")


def cc_csr(n: int, offsets, cols, variant=None, stream=None):
    """Canonical labels from CSR; int32/uint32 offsets select gconn_cc_csr32."""
    torch = _torch()
    labels = torch.empty(n, dtype=torch.int32, device=offsets.device)
    if _off32(offsets):
        gconn_cc_csr32(n, offsets, cols, labels, variant, stream)  # noqa: F405
    else:
        gconn_cc_csr(n, offsets, cols, labels, variant, stream)  # noqa: F405
    return labels


def spanning_forest(n: int, edges, variant=None, stream=None, labels: bool = False):
    """(forest edge ids int64[count], labels or None) for a COO edge list."""
    torch = _torch()
    dev = edges.device
    forest = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev) if labels else None
    gconn_spanning_forest(n, int(edges.shape[0]), edges, forest, count, lab, variant, stream)  # noqa: F405
    c = int(count.item())
    return forest[:c], lab


def spanning_forest_csr(n: int, offsets, cols, variant=None, stream=None, labels: bool = False):
    """(forest arc positions int64[count], labels or None) for CSR input."""
    torch = _torch()
    dev = offsets.device
    forest = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev) if labels else None
    fn = gconn_spanning_forest_csr32 if _off32(offsets) else gconn_spanning_forest_csr  # noqa: F405
    fn(n, offsets, cols, forest, count, lab, variant, stream)
    c = int(count.item())
    return forest[:c], lab


class Incremental:
    """Device-resident incremental connectivity (Section 3.5)."""

    def __init__(self, n: int, variant=None, stream=None):
        self.n = n
        self.stream = stream
        self.h = gconn_inc_create(n, variant, stream)  # noqa: F405

    def insert(self, edges, stream=None):
        gconn_inc_insert_batch(self.h, int(edges.shape[0]), edges, stream or self.stream)  # noqa: F405

    def query(self, pairs, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty(int(pairs.shape[0]), dtype=torch.uint8, device=pairs.device)
        gconn_inc_query(self.h, int(pairs.shape[0]), pairs, out, stream or self.stream)  # noqa: F405
        return out

    def edges_inspected(self):
        """(edge inspections of the last insert batch, total) -- Section 4.4."""
        return gconn_inc_edges_inspected(self.h)  # noqa: F405

    def labels(self, device=None, stream=None):
        torch = _torch()
        out = torch.empty(self.n, dtype=torch.int32, device=device or "cuda")
        gconn_inc_labels(self.h, out, stream or self.stream)  # noqa: F405
        return out

    def close(self):
        if self.h is not None and self.h.value:
            gconn_inc_destroy(self.h)  # noqa: F405
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
