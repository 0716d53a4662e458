"""gconn_cc_csr_noalloc: the connected-components call for callers that may
not allocate device memory (another allocator owns the GPU, or a fixed memory
budget forbids new allocations).  It must give exactly the labels of the
allocating gconn_cc_csr on the same inputs, call after call, even though
every call reuses one fixed scratch array inside the library.

This file is collected last on purpose: a run that stops at the first
failure has then already run every other test."""
import numpy as np
import pytest

import graphgen
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


def test_noalloc_matches_allocating_call_twice():
    """Two calls in a row, on different graphs (the second must not see the
    first call's leftovers), each bit-exact with gconn_cc_csr."""
    n1 = 1 << 16
    e1 = graphgen.rmat(16, 600_001, 21)
    n2 = 100_003
    e2 = graphgen.er(n2, 70_001, 22)
    cases = [(n1, e1, g.make_variant(sample="kout", link="remcas", splice="split_one")),
             (n2, e2, g.make_variant(sample="kout", link="remcas", splice="split_one"))]
    for n, e, v in cases:
        off, cols = graphgen.csr(n, e)
        a, b = _both(n, off, cols, v)
        assert (a == b).all()


def test_noalloc_other_variants_and_no_memory_growth():
    import torch
    n = 1 << 15
    e = graphgen.rmat(15, 200_000, 5)
    off, cols = graphgen.csr(n, e)
    d_off, d_cols = dev(off), dev(cols)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    v0 = g.make_variant(sample="hb", link="async", find="compress")
    ref = torch.empty(n, dtype=torch.int32, device="cuda")
    g.gconn_cc_csr_noalloc(n, d_off, d_cols, out, v0)          # set-up done on the first call
    g.gconn_sync()
    for spec in [dict(sample="none", link="early"), dict(sample="kout", link="async", find="halve"),
                 dict(sample="hb", link="remcas", find="split", splice="halve_one")]:
        v = g.make_variant(**spec)
        # the first launch of a kernel lets the driver load its code (lazy
        # module loading); what must not grow is memory across repeat calls
        g.gconn_cc_csr_noalloc(n, d_off, d_cols, out, v)
        g.gconn_sync()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        g.gconn_cc_csr_noalloc(n, d_off, d_cols, out, v)
        g.gconn_sync()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0             # no device allocation
        got = host_u32(out)
        g.gconn_cc_csr(n, d_off, d_cols, ref, v)
        g.gconn_sync()
        assert (got == host_u32(ref)).all(), spec


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
