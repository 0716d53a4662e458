"""Pins for the seeded input generators (graphgen): published SplitMix64
outputs, determinism, distributions, and the COO -> CSR builder."""
import numpy as np

import graphgen


def test_splitmix64_published_outputs():
    # First outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014;
    # the reference vectors distributed with the algorithm).
    assert graphgen.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF
    assert graphgen.splitmix64_at(0, 1) == 0x6E789E6AA1B965F4
    assert graphgen.splitmix64_at(0, 2) == 0x06C45D188009454F


def test_hash_fill_is_counter_based():
    a = graphgen.hash_fill(5, 3, 0, 1000)
    b = graphgen.hash_fill(5, 3, 400, 100)
    assert (a[400:500] == b).all()
    base = graphgen.stream_base(5, 3)
    assert int(a[7]) == graphgen.splitmix64_at(base, 7)


def test_generators_deterministic_and_seeded():
    assert (graphgen.er(1000, 5000, 1) == graphgen.er(1000, 5000, 1)).all()
    assert not (graphgen.er(1000, 5000, 1) == graphgen.er(1000, 5000, 2)).all()
    assert (graphgen.rmat(12, 5000, 3) == graphgen.rmat(12, 5000, 3)).all()
    e = graphgen.rmat(12, 3000, 3)
    r = graphgen.rmat_range(12, 1000, 500, 3, perm=graphgen.permutation(1 << 12, 3, 6))
    assert (e[1000:1500] == r).all()


def test_er_uniform_range():
    e = graphgen.er(100, 200000, 8)
    assert e.max() < 100
    cnt = np.bincount(e.ravel(), minlength=100)
    assert abs(cnt.mean() - 4000) < 1 and cnt.min() > 3600 and cnt.max() < 4400


def test_rmat_quadrant_probabilities():
    # scale 1: one draw per edge, so the quadrant frequencies are a, b, c, d
    e = graphgen.rmat(1, 400000, 4, permute=False)
    q = e[:, 0] * 2 + e[:, 1]
    freq = np.bincount(q, minlength=4) / len(q)
    assert np.allclose(freq, [0.57, 0.19, 0.19, 0.05], atol=0.004)
    e = graphgen.rmat(10, 50000, 4, permute=False)
    assert e.max() < 1024


def test_permutation_is_permutation():
    p = graphgen.permutation(100000, 9)
    assert (np.sort(p) == np.arange(100000)).all()
    assert not (p == np.arange(100000)).all()


def test_grid_paths_structure():
    side, npaths, plen = 50, 5, 40
    n, e = graphgen.grid_paths(side, 0.0, npaths, plen, 2)
    assert n == side * side + npaths * plen
    assert len(e) == 2 * side * (side - 1) + npaths * (plen - 1)
    n2, e2 = graphgen.grid_paths(side, 0.05, npaths, plen, 2)
    kept = len(e2) - npaths * (plen - 1)
    assert abs(kept / (2 * side * (side - 1)) - 0.95) < 0.02
    grid = e[(e < side * side).all(1)]
    d = np.abs(grid[:, 0].astype(int) - grid[:, 1].astype(int))
    assert set(np.unique(d).tolist()) == {1, side}


def test_batched_sizes():
    vo, eo, e = graphgen.batched(200, 5)
    n = np.diff(vo)
    m = np.diff(eo)
    assert n.min() >= 256 and n.max() <= 65536
    assert (m >= 2 * n - 1).all() and (m <= 16 * n + 1).all()
    for g in range(0, 200, 17):
        sub = e[int(eo[g]):int(eo[g + 1])]
        assert sub.max() < n[g]


def test_csr_roundtrip():
    n = 3000
    e = graphgen.er(n, 10000, 12)
    off, cols = graphgen.csr(n, e)
    assert off[0] == 0 and off[-1] == 2 * len(e)
    rows = np.repeat(np.arange(n), np.diff(off).astype(np.int64))
    arcs = sorted(zip(rows.tolist(), cols.tolist()))
    want = sorted([(int(u), int(v)) for u, v in e] + [(int(v), int(u)) for u, v in e])
    assert arcs == want
    for v in range(0, n, 97):
        r = cols[off[v]:off[v + 1]]
        assert (np.diff(r.astype(np.int64)) >= 0).all()


def test_ba_endpoint_copying_and_shape():
    """Barabasi-Albert by Batagelj-Brandes endpoint copying: edge e starts at
    e // d, its far end copies a uniformly drawn earlier endpoint (so it is an
    earlier-or-same vertex), and the degree distribution is heavy-tailed."""
    n, d, seed = 2000, 3, 41
    e = graphgen.ba(n, d, seed)
    m = n * d
    assert e.shape == (m, 2)
    assert (e[:, 0] == np.arange(m) // d).all()
    assert (e[:, 1] <= e[:, 0]).all()
    # the copying rule, restated from the published method on the same draws
    h = graphgen.hash_fill(seed, 9, 0, m)
    flat = np.empty(2 * m, np.int64)
    for i in range(m):
        flat[2 * i] = i // d
        r = (int(h[i]) * (2 * i + 1)) >> 64
        flat[2 * i + 1] = flat[r]
    assert (flat.reshape(m, 2) == e).all()
    assert (graphgen.ba(n, d, seed) == e).all() and not (graphgen.ba(n, d, seed + 1) == e).all()
    big = graphgen.ba(100_000, 4, 5)
    deg = np.bincount(big.ravel(), minlength=100_000)
    assert deg.max() > 20 * deg.mean()          # hubs: early vertices gather ~ d sqrt(n / i) edges


def test_generator_outputs_are_stable():
    """Every generator's output for a fixed seed, pinned by hash: the inputs the
    tests and the benchmark use must not drift between builds or machines (the
    C code depends on no platform integer width beyond uint64 / __int128)."""
    import hashlib

    def h(a):
        return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:16]
    assert h(graphgen.er(1000, 5000, 1)) == "86c9ca8de9ccff49"
    assert h(graphgen.rmat(12, 5000, 3)) == "6de8fdc2613d7e8a"
    assert h(graphgen.permutation(1 << 12, 3, 6)) == "5e4ce5916122c76a"
    n, e = graphgen.grid_paths(16, 0.05, 4, 64, 7)
    assert n == 512 and h(e) == "d8ffa09ca42169d2"
    assert h(graphgen.pairs_range(1000, 0, 4000, 9)) == "403c3d91c30db885"
    assert h(graphgen.ba(2000, 4, 11)) == "45108feb8c446438"
    assert [h(x) for x in graphgen.batched(8, 5, nmin=16, nmax=256)] == \
        ["dccbdf458f5f2de6", "04b766d1c5298541", "d29b29b0103d69c9"]
