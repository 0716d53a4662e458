"""The multicore CPU baseline (bench.py's comparison leg) reaches the
oracle's canonical labels on every input shape, with one and several threads."""
import numpy as np
import pytest

import cpu_baseline
import graphgen
import oracle


def _graphs():
    yield "empty", 10, np.zeros((0, 2), np.uint32)
    yield "selfloops", 6, np.array([[i, i] for i in range(6)], np.uint32)
    yield "path", 50, np.array([[i, i + 1] for i in range(49)], np.uint32)
    yield "er", 3000, graphgen.er(3000, 4000, 11)
    yield "rmat", 1 << 12, graphgen.rmat(12, 30_000, 12)
    n, e = graphgen.grid_paths(32, 0.05, 4, 64, 13)
    yield "grid_paths", n, e


@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("k", [1, 2, 5])
def test_multicore_baseline_matches_oracle(threads, k):
    for name, n, e in _graphs():
        off, cols = graphgen.csr(n, e)
        lab = cpu_baseline.cc_csr(n, off, cols, k=k, threads=threads)
        assert (lab == oracle.cc_uf(n, e)).all(), name


def test_multicore_baseline_range_error():
    off = np.array([0, 1, 1], np.uint64)
    cols = np.array([7], np.uint32)
    with pytest.raises(ValueError):
        cpu_baseline.cc_csr(2, off, cols)
