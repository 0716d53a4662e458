"""Host logic of the benchmark's serving leg: the parallel RMAT stream equals
the serial generator's output, and the serving trace alternates insert and
query batches of the law's sizes that cover each session's stream."""
import numpy as np

import bench
import graphgen


def test_parallel_rmat_stream_equals_serial():
    n_scale, total, seed = 12, 100_003, 77
    perm = graphgen.permutation(1 << n_scale, seed, 6)
    par = bench.rmat_stream(n_scale, total, seed, perm, threads=7)
    ser = graphgen.rmat_range(n_scale, 0, total, seed, perm=perm)
    assert par.shape == (total, 2) and np.array_equal(par, ser)


def test_serving_trace_shape():
    total = 50_000
    n, trace, answers = bench.serving_trace(2, 12, total, 99)
    assert n == 1 << 12 and len(trace) == 2
    for s, reqs in enumerate(trace):
        ops = [op for op, _, _ in reqs]
        assert ops == [0, 1] * (len(reqs) // 2)
        sizes = [len(a) for _, a, _ in reqs[::2]]
        assert sizes == [len(a) for _, a, _ in reqs[1::2]] == bench.inc_batches(99 + s, total)
        assert sum(sizes) == total
        assert all(s_ >= 1000 for s_ in sizes[:-1])
        ins = np.concatenate([a for op, a, _ in reqs if op == 0])
        assert np.array_equal(ins, bench.rmat_stream(12, total, 99 + s, graphgen.permutation(1 << 12, 99, 6)))
