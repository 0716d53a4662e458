"""The benchmark's algorithmic-bytes model: the per-unit terms of the
method's measurement model (init 4n, k-out sampling 4(n+1) + 4kn, vertex
gathering 4n, CSR finish 4 * active arcs + 8 * active vertices, finalisation
8n, COO finish 8m), checked on numbers worked out by hand."""
import bench


def test_static_pass_terms_rmat_s22():
    n, m = 1 << 22, 1 << 26
    st = {"n": n, "m": m, "k": 2, "active_vertices": 1544, "active_arcs": 5000}
    assert bench.alg_bytes("init", st) == 16_777_216
    assert bench.alg_bytes("kout", st) == 4 * (n + 1) + 8 * n == 50_331_652
    assert bench.alg_bytes("vg", st) == 16_777_216
    assert bench.alg_bytes("finish", st) == 4 * 5000 + 8 * 1544
    assert bench.alg_bytes("finalize", st) == 33_554_432
    assert bench.alg_bytes("union_coo", st) == 8 * m
    assert bench.alg_bytes("kout_deferred", st) is None
    whole = sum(bench.alg_bytes(k, st) for k in ("init", "kout", "vg", "finish", "finalize"))
    assert whole == 117_440_516 + 4 * 5000 + 8 * 1544


def test_roofline_fraction():
    r = bench.roofline(117_440_516, 0.1, 6770.5, "measured", kernel="pass")
    assert r["achieved"] == round(117_440_516 / 1e-4 / 1e9, 1)
    assert abs(r["frac"] - 1174.40516 / 6770.5) < 1e-4
    assert r["unit"] == "GB/s" and r["bound"] == "hbm" and r["kernel"] == "pass"

