"""GPU parity at the largest vertex count the ABI accepts, n = 0xFFFFFFFE
(ids up to 0xFFFFFFFD; 0xFFFFFFFF is reserved).  The edges touch a few ids at
both ends of the range and around 2^31, so labels above 2^31 are read back,
every per-vertex loop runs past 2^32 - 2^10 and every 64-bit index path is
taken.  The oracle runs on the touched ids, relabelled in increasing order
(which keeps each component's minimum); every other vertex must keep its own
id, checked on the device in chunks.

Device memory: the COO and incremental cases hold about 40 GB, the CSR case
about 130 GB (offsets 32 GB, labels and parents 16 GB each, the gathering
lists 64 GB), all returned after each test."""
import numpy as np
import pytest

import oracle
import paper_2008_11839_gb300 as g

pytestmark = pytest.mark.gpu

N_MAX = 0xFFFFFFFE
CHUNK = 1 << 28


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g.build()
    g.lib()


@pytest.fixture(autouse=True)
def _release():
    yield
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    g.gconn_release_cached()


def _edges(n):
    top = [n - 1, n - 2, n - 3, n - 4, n - 5, n - 33, n - 34]
    mid = [(1 << 31) - 1, 1 << 31, (1 << 31) + 1, 3 << 30]
    e = [(top[0], top[1]), (top[1], top[4]),               # component {n-5, n-2, n-1}: label above 2^31
         (top[2], mid[1]), (mid[1], 7),                     # {7, 2^31, n-3}
         (top[3], top[3]),                                  # a self-loop only
         (top[5], top[6]), (top[6], top[5]),                # a duplicate pair
         (0, 1), (1, mid[0]), (mid[0], top[6]),             # {0, 1, 2^31-1, n-34, n-33}
         (100, mid[3]), (mid[3], mid[2])]                   # {100, 2^31+1, 3*2^30}
    return np.array(e, dtype=np.uint64).astype(np.uint32)


def _expected(edges):
    """Touched ids (ascending) and their oracle labels."""
    t = np.unique(edges.astype(np.uint64))
    local = np.searchsorted(t, edges.astype(np.uint64)).astype(np.uint32)
    return t, t[oracle.cc_uf(len(t), local)].astype(np.uint64)


def _check(labels, n, touched, want):
    import torch
    idx = torch.from_numpy(touched.astype(np.int64)).cuda()
    got = (labels[idx].to(torch.int64) & 0xFFFFFFFF).cpu().numpy().astype(np.uint64)
    assert (got == want).all(), (got, want)
    for s in range(0, n, CHUNK):
        e = min(n, s + CHUNK)
        x = labels[s:e].to(torch.int64) & 0xFFFFFFFF
        ar = torch.arange(s, e, dtype=torch.int64, device="cuda")
        inside = touched[(touched >= s) & (touched < e)].astype(np.int64) - s
        if len(inside):
            ti = torch.from_numpy(inside).cuda()
            x[ti] = ar[ti]
        assert torch.equal(x, ar), f"untouched vertices relabelled in [{s}, {e})"
        del x, ar


def _dev_edges(e):
    import torch
    return torch.from_numpy(e.view(np.int32)).cuda()


def test_coo_at_maximum_n():
    import torch
    e = _edges(N_MAX)
    touched, want = _expected(e)
    labels = torch.empty(N_MAX, dtype=torch.int32, device="cuda")
    g.gconn_cc(N_MAX, len(e), _dev_edges(e), labels, g.make_variant(link="remcas", splice="split_one"))
    g.gconn_sync()
    _check(labels, N_MAX, touched, want)


def test_csr_kout_at_maximum_n():
    import torch
    e = _edges(N_MAX).astype(np.uint64)
    arcs = np.unique(np.concatenate([e, e[:, ::-1]]), axis=0)   # rows, then columns ascending
    rows = torch.from_numpy(arcs[:, 0].astype(np.int64)).cuda()
    cols = torch.from_numpy(arcs[:, 1].astype(np.uint32).view(np.int32)).cuda()
    off = torch.empty(N_MAX + 1, dtype=torch.int64, device="cuda")
    for s in range(0, N_MAX + 1, CHUNK):
        t = min(N_MAX + 1, s + CHUNK)
        off[s:t] = torch.searchsorted(rows, torch.arange(s, t, dtype=torch.int64, device="cuda"))
    assert int(off[-1]) == len(arcs)
    touched, want = _expected(_edges(N_MAX))
    labels = torch.empty(N_MAX, dtype=torch.int32, device="cuda")
    g.gconn_cc_csr(N_MAX, off, cols, labels, g.make_variant(sample="kout", link="remcas", splice="split_one"))
    g.gconn_sync()
    _check(labels, N_MAX, touched, want)


def test_incremental_at_maximum_n():
    import torch
    e = _edges(N_MAX)
    touched, want = _expected(e)
    inc = g.Incremental(N_MAX, g.make_variant(link="early"))
    try:
        inc.insert(_dev_edges(e[:6]))
        inc.insert(_dev_edges(e[6:]))
        lab_of = dict(zip(touched.tolist(), want.tolist()))
        q = np.array([(N_MAX - 1, N_MAX - 5), (N_MAX - 3, 7), (N_MAX - 33, 0), (N_MAX - 4, N_MAX - 5),
                      (N_MAX - 1, 0), (5, 6), (N_MAX - 1, N_MAX - 1)], dtype=np.uint64).astype(np.uint32)
        got = inc.query(_dev_edges(q)).cpu().numpy()
        exp = [lab_of.get(int(a), int(a)) == lab_of.get(int(b), int(b)) for a, b in q]
        assert got.astype(bool).tolist() == exp
        labels = inc.labels()
        g.gconn_sync()
        _check(labels, N_MAX, touched, want)
    finally:
        inc.close()
