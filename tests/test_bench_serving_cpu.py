"""Host logic of the benchmark's serving leg: the parallel RMAT stream equals
the serial generator's output, and the serving trace alternates insert and
query batches of the law's sizes that cover each session's stream, and the
open-loop driver runs both drivers over pooled arrival draws with identical
answers (against a host stand-in for the library)."""
import types

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


class _FakeLib:
    """The serving leg's calls on the host: a union-find per handle / session;
    the server runs each request at submission.  Stands in for the library so
    that the open-loop driver (arrivals, threads, pooled draws, answer checks)
    runs without a GPU."""
    GCONN_OP_INSERT, GCONN_OP_QUERY = 0, 1

    class _UF:
        def __init__(self, n):
            self.p = np.arange(n, dtype=np.int64)

        def find(self, x):
            p = self.p
            while p[x] != x:
                p[x] = p[p[x]]
                x = p[x]
            return x

        def insert(self, pairs):
            for u, v in pairs:
                a, b = self.find(int(u)), self.find(int(v))
                if a != b:
                    self.p[max(a, b)] = min(a, b)

        def query(self, pairs, out):
            out[:] = [self.find(int(u)) == self.find(int(v)) for u, v in pairs]

    def __init__(self):
        self.submits = 0

    def make_variant(self, **kw):
        return None

    def gconn_inc_create(self, n, v):
        return self._UF(n)

    def gconn_inc_insert_batch(self, h, m, a):
        h.insert(a[:m])

    def gconn_inc_query(self, h, q, a, out):
        h.query(a[:q], out)

    def gconn_inc_destroy(self, h):
        pass

    def gconn_server_create(self):
        return {"sessions": [], "done": {}}

    def gconn_server_open_session(self, srv, n, v):
        srv["sessions"].append(self._UF(n))
        return len(srv["sessions"]) - 1

    def gconn_server_submit(self, srv, sid, op, count, pairs, result):
        uf = srv["sessions"][sid]
        if op == self.GCONN_OP_INSERT:
            uf.insert(pairs[:count])
        else:
            uf.query(pairs[:count], result)
        self.submits += 1
        t = len(srv["done"])
        srv["done"][t] = 0.01
        return t

    def gconn_server_wait(self, srv, t):
        return srv["done"][t]

    def gconn_server_stats(self, srv):
        return {"launches": len(srv["done"]), "groups": len(srv["done"])}

    def gconn_server_destroy(self, srv):
        pass


def test_open_loop_driver_pools_draws(monkeypatch):
    monkeypatch.setattr(bench, "host_array", lambda shape, dtype, pinned: np.empty(shape, dtype))
    lib = _FakeLib()
    torch_stub = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    res = bench.run_serving(lib, torch_stub, None, 2, 4_000, 10, (3.0, 3.3), [0.5, 1.0], reps=3)
    assert res["identical_answers"] and res["ops"] == 2 * 2 * 4_000
    nreq = res["requests"]
    assert lib.submits == 2 * 3 * nreq               # two loads, three draws each
    for row in res["loads"]:
        assert row["identical_answers"]
        assert len(row["p50_plain_served_per_draw"]) == 3
        assert row["served"]["launches"] == 3 * nreq
        assert row["plain"]["latency_ms_p50"] >= 0 and row["served"]["latency_ms_p99"] >= 0
