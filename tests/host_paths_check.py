"""Host-buffer calls checked against the oracle (run as a child process by
tests/test_gpu_host_paths.py, once with host inputs read in place and once
with GCONN_HOST_STAGE=1, which makes the library copy them)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402
import paper_2008_11839_gb300 as g  # noqa: E402


def main():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.init()
    n = 40_009
    e = graphgen.rmat(16, 300_000, 41) % np.uint32(n)
    e = np.ascontiguousarray(e.astype(np.uint32))
    ref = oracle.cc_uf(n, e)
    off, cols = graphgen.csr(n, e)
    # static CSR, uint64 and uint32 offsets, pageable and page-locked inputs
    for pinned in (False, True):
        cols_h = torch.from_numpy(cols.view(np.int32)).pin_memory().numpy().view(np.uint32) if pinned else cols
        for o in (off, off.astype(np.uint32)):
            out = np.empty(n, np.uint32)
            fn = g.gconn_cc_csr32 if o.dtype == np.uint32 else g.gconn_cc_csr
            fn(n, o, cols_h, out, g.make_variant(sample="kout", link="remcas", splice="split_one"))
            assert (out == ref).all(), ("csr", pinned, o.dtype)
    # static COO (a one-pass finish reads the edges in place; SV re-reads them)
    for v in (g.make_variant(link="remcas", splice="split_one"), g.make_variant(link="sv")):
        out = np.empty(n, np.uint32)
        g.gconn_cc(n, len(e), e, out, v)
        assert (out == ref).all(), "coo"
    # incremental batches and queries with host buffers
    inc = oracle.Incremental(n)
    h = g.gconn_inc_create(n, g.make_variant(link="early"))
    for k in range(4):
        b = e[k * 50_000:(k + 1) * 50_000]
        q = graphgen.pairs_range(n, k * 50_000, 50_000, 43)
        g.gconn_inc_insert_batch(h, len(b), b)
        inc.insert(b)
        got = np.empty(len(q), np.uint8)
        g.gconn_inc_query(h, len(q), q, got)
        assert (got == inc.query(q)).all(), ("inc", k)
    g.gconn_inc_destroy(h)
    # the serving loop: small requests merge, the big one too where in place
    srv = g.gconn_server_create()
    sid = g.gconn_server_open_session(srv, n, g.make_variant(link="early"))
    inc = oracle.Incremental(n)
    tickets, checks = [], []
    for k, c in enumerate([100, 3000, 5_000_000, 700]):
        b = graphgen.rmat_range(16, k << 24, c, 45) % np.uint32(n)
        b = np.ascontiguousarray(b.astype(np.uint32))
        q = graphgen.pairs_range(n, k << 24, c, 47)
        res = np.empty(c, np.uint8)
        tickets.append(g.gconn_server_submit(srv, sid, g.GCONN_OP_INSERT, c, b, None))
        tickets.append(g.gconn_server_submit(srv, sid, g.GCONN_OP_QUERY, c, q, res))
        inc.insert(b)
        checks.append((res, inc.query(q), b, q))
    for t in tickets:
        g.gconn_server_wait(srv, t)
    for res, want, _, _ in checks:
        assert (res == want).all(), "serve"
    lab = np.empty(n, np.uint32)
    g.gconn_server_labels(srv, sid, lab)
    assert (lab == inc.labels()).all()
    g.gconn_server_destroy(srv)
    print("host paths ok", os.environ.get("GCONN_HOST_STAGE", "0"))


if __name__ == "__main__":
    main()
