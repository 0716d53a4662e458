"""gconn_cc_csr_noalloc: the connected-components call for callers that may
not allocate device memory (another allocator owns the GPU, or a fixed memory
budget forbids new allocations).  It must give exactly the canonical labels
of the oracle -- and so of the allocating gconn_cc_csr -- on the same inputs,
call after call, even though every call reuses one fixed scratch array
inside the library.

This file is collected last on purpose: a run that stops at the first
failure has then already run every other test."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2008_11839_gb300 as g
from gpu_util import dev, host_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g.build()


def _both(n, off, cols, v):
    import torch
    d_off, d_cols = dev(off), dev(cols)
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    b = torch.empty(n, dtype=torch.int32, device="cuda")
    g.gconn_cc_csr_noalloc(n, d_off, d_cols, a, v)
    g.gconn_sync()
    g.gconn_cc_csr(n, d_off, d_cols, b, v)
    g.gconn_sync()
    return host_u32(a), host_u32(b)


def test_noalloc_matches_oracle_twice():
    """Two calls in a row, on different graphs (the second must not see the
    first call's leftovers), each bit-exact with the oracle and with
    gconn_cc_csr."""
    n1 = 1 << 16
    e1 = graphgen.rmat(16, 600_001, 21)
    n2 = 100_003
    e2 = graphgen.er(n2, 70_001, 22)
    v = g.make_variant(sample="kout", link="remcas", splice="split_one")
    for n, e in [(n1, e1), (n2, e2)]:
        off, cols = graphgen.csr(n, e)
        a, b = _both(n, off, cols, v)
        ref = oracle.cc_uf(n, e)
        assert (a == ref).all()
        assert (b == ref).all()


def test_noalloc_takes_no_memory_after_setup():
    """After the set-up call (n == 0), no call takes device memory -- not even
    the first call of a variant that has not run yet."""
    import torch
    n = 1 << 15
    e = graphgen.rmat(15, 200_000, 5)
    ref = oracle.cc_uf(n, e)
    off, cols = graphgen.csr(n, e)
    d_off, d_cols = dev(off), dev(cols)
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4)]
    specs = [dict(sample="hb", link="async", find="compress"), dict(sample="none", link="early"),
             dict(sample="kout", link="async", find="halve"),
             dict(sample="hb", link="remcas", find="split", splice="halve_one")]
    g.gconn_cc_csr_noalloc(0, None, None, None)                 # set-up only
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for out, spec in zip(outs, specs):
        g.gconn_cc_csr_noalloc(n, d_off, d_cols, out, g.make_variant(**spec))
        torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    g.gconn_sync()
    assert free1 == free0, f"device memory fell by {free0 - free1} bytes"
    for out, spec in zip(outs, specs):
        assert (host_u32(out) == ref).all(), spec


def test_noalloc_max_n_on_a_stream():
    """n = GCONN_NOALLOC_MAX_N, k-out sampling, on a non-default stream."""
    import torch
    n = g.GCONN_NOALLOC_MAX_N
    e = graphgen.rmat(20, 1 << 23, 23)
    off, cols = graphgen.csr(n, e)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        d_off, d_cols = dev(off), dev(cols)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
    g.gconn_cc_csr_noalloc(n, d_off, d_cols, out, g.make_variant(sample="kout", link="remcas", splice="split_one"),
                           st)
    g.gconn_sync(st)
    assert (host_u32(out) == oracle.cc_uf(n, e)).all()


def _circulant_with_hubs(n, width, hubs, hub_deg, seed):
    """Every vertex joined to the next `width` ids (degree 2 * width), plus
    `hubs` vertices with `hub_deg` extra edges each to seeded vertices."""
    v = np.arange(n, dtype=np.uint64)
    ring = [np.stack([v, (v + k) % n], 1) for k in range(1, width + 1)]
    h = graphgen.hash_fill(seed, 3, 0, hubs * hub_deg).astype(np.uint64)
    tgt = ((h >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    src = np.repeat(np.arange(hubs, dtype=np.uint64) * (n // hubs) + n // (2 * hubs), hub_deg)
    e = np.concatenate(ring + [np.stack([src, tgt], 1)]).astype(np.uint32)
    return e


def test_noalloc_task_list_overflow():
    """More warp tasks than the fixed task list holds: every vertex has degree
    34 (> the thread-per-vertex limit, one 256-arc task each) and four hubs
    add 2,052 tasks, 1,024 beyond the list's capacity of n + 1,024, so the
    vertices that reserve last go to the overflow list.  n is the maximum."""
    n = g.GCONN_NOALLOC_MAX_N
    e = _circulant_with_hubs(n, 17, 4, 131_072, 24)
    off, cols = graphgen.csr(n, e)
    deg = np.diff(off.astype(np.int64))
    tasks = int(((deg + 255) // 256)[deg > 32].sum())
    assert tasks > n + 1024                                     # the overflow list is reached
    ref = oracle.cc_uf(n, e)
    for spec in [dict(sample="none", link="remcas", splice="split_one"), dict(sample="none", link="async")]:
        a, b = _both(n, off, cols, g.make_variant(**spec))
        assert (a == ref).all(), spec
        assert (b == ref).all(), spec


def test_noalloc_rejects_what_it_cannot_do():
    import torch
    n = g.GCONN_NOALLOC_MAX_N + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GconnError) as ex:
        g.gconn_cc_csr_noalloc(n, off, out, out)
    assert ex.value.status == g.GCONN_E_INVAL
    small_off = np.zeros(11, np.uint64)
    with pytest.raises(g.GconnError) as ex:                      # host buffers would need staging
        g.gconn_cc_csr_noalloc(10, small_off, np.zeros(1, np.uint32), np.empty(10, np.uint32))
    assert ex.value.status == g.GCONN_E_INVAL
    d_off = dev(small_off)
    with pytest.raises(g.GconnError) as ex:
        g.gconn_cc_csr_noalloc(10, d_off, out, out, g.make_variant(sample="bfs"))
    assert ex.value.status == g.GCONN_E_UNSUPPORTED
