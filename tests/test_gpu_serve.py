"""The serving loop: every session's answers are the same when it runs alone
and when it runs mixed with other sessions submitting concurrently, and both
equal the sequential oracle replay (Section 3.5 semantics)."""
import threading

import numpy as np
import pytest

import graphgen
import oracle
import paper_2008_11839_gb300 as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g.build()


def _session_stream(n, seed, nreq=40):
    """Alternating-ish insert / query requests of random sizes (host arrays)."""
    rng = np.random.default_rng(seed)
    scale = int(np.ceil(np.log2(n)))
    perm = graphgen.permutation(1 << scale, seed, 6)
    reqs, ins_pos, q_pos = [], 0, 0
    for _ in range(nreq):
        c = int(rng.integers(1, 6000))
        if rng.random() < 0.5:
            e = graphgen.rmat_range(scale, ins_pos, c, seed, perm=perm) % np.uint32(n)
            ins_pos += c
            reqs.append((g.GCONN_OP_INSERT, np.ascontiguousarray(e)))
        else:
            p = graphgen.pairs_range(n, q_pos, c, seed)
            q_pos += c
            reqs.append((g.GCONN_OP_QUERY, p))
    return reqs


def _oracle_answers(n, reqs):
    inc = oracle.Incremental(n)
    out = []
    for op, arr in reqs:
        if op == g.GCONN_OP_INSERT:
            inc.insert(arr)
            out.append(None)
        else:
            out.append(inc.query(arr))
    return out, inc.labels()


def _run(server, sid, reqs):
    tickets, results = [], []
    for op, arr in reqs:
        res = np.empty(len(arr), np.uint8) if op == g.GCONN_OP_QUERY else None
        tickets.append(g.gconn_server_submit(server, sid, op, len(arr), arr, res))
        results.append(res)
    lat = [g.gconn_server_wait(server, t) for t in tickets]
    return results, lat


SESSIONS = [(3000, 1, dict(link="early")), (20000, 2, dict(link="async", find="halve")),
            (7000, 3, dict(link="remcas", splice="splice")), (50000, 4, dict(link="jtb")),
            (12000, 5, dict(link="lt", lt="PRF")), (9000, 6, dict(link="sv"))]


def test_alone_equals_mixed_equals_oracle():
    streams = [_session_stream(n, seed) for n, seed, _ in SESSIONS]
    refs = [_oracle_answers(n, s) for (n, _, _), s in zip(SESSIONS, streams)]
    # alone: one server per session
    alone = []
    for (n, seed, kw), reqs in zip(SESSIONS, streams):
        srv = g.gconn_server_create()
        sid = g.gconn_server_open_session(srv, n, g.make_variant(**kw))
        res, _ = _run(srv, sid, reqs)
        lab = np.empty(n, np.uint32)
        g.gconn_server_labels(srv, sid, lab)
        g.gconn_server_destroy(srv)
        alone.append((res, lab))
    # mixed: one server, every session submitting from its own thread
    cfg = g.gconn_server_config_default()
    cfg.slots = 4
    srv = g.gconn_server_create(cfg)
    sids = [g.gconn_server_open_session(srv, n, g.make_variant(**kw)) for n, _, kw in SESSIONS]
    mixed = [None] * len(SESSIONS)

    def worker(i):
        mixed[i] = _run(srv, sids[i], streams[i])
    th = [threading.Thread(target=worker, args=(i,)) for i in range(len(SESSIONS))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i, (n, _, _) in enumerate(SESSIONS):
        lab = np.empty(n, np.uint32)
        g.gconn_server_labels(srv, sids[i], lab)
        ref_ans, ref_lab = refs[i]
        a_res, a_lab = alone[i]
        m_res, _ = mixed[i]
        for ra, rm, rr in zip(a_res, m_res, ref_ans):
            if rr is None:
                continue
            assert (ra == rr).all() and (rm == rr).all()
        assert (a_lab == ref_lab).all() and (lab == ref_lab).all()
    stats = g.gconn_server_stats(srv)
    assert stats["requests"] >= sum(len(s) for s in streams)
    g.gconn_server_destroy(srv)


def test_coalescing_and_tiny_budget():
    n = 4000
    reqs = [(g.GCONN_OP_INSERT, graphgen.er(n, 50, 100 + i)) for i in range(200)]
    reqs.append((g.GCONN_OP_QUERY, graphgen.pairs_range(n, 0, 3000, 9)))
    cfg = g.gconn_server_config_default()
    cfg.slots = 1
    srv = g.gconn_server_create(cfg)
    sid = g.gconn_server_open_session(srv, n)
    res, lat = _run(srv, sid, reqs)
    allins = np.concatenate([a for op, a in reqs if op == g.GCONN_OP_INSERT])
    ref = oracle.cc_uf(n, allins)
    q = reqs[-1][1]
    assert (res[-1] == (ref[q[:, 0]] == ref[q[:, 1]])).all()
    st = g.gconn_server_stats(srv)
    assert st["groups"] < st["requests"]                 # small requests were merged
    assert all(x >= 0 for x in lat)
    g.gconn_server_destroy(srv)
    # a budget smaller than any request: requests still run, one at a time
    cfg.device_budget_bytes = 64
    cfg.slots = 2
    srv = g.gconn_server_create(cfg)
    sid = g.gconn_server_open_session(srv, n)
    res2, _ = _run(srv, sid, reqs)
    assert (res2[-1] == res[-1]).all()
    g.gconn_server_destroy(srv)


def test_errors():
    srv = g.gconn_server_create()
    sid = g.gconn_server_open_session(srv, 100)
    with pytest.raises(g.GconnError):
        g.gconn_server_submit(srv, sid + 99, g.GCONN_OP_INSERT, 1, np.array([[0, 1]], np.uint32))
    t = g.gconn_server_submit(srv, sid, g.GCONN_OP_INSERT, 1, np.array([[0, 100]], np.uint32))
    with pytest.raises(g.GconnError) as ex:
        g.gconn_server_wait(srv, t)
    assert ex.value.status == g.GCONN_E_RANGE
    ok = g.gconn_server_submit(srv, sid, g.GCONN_OP_INSERT, 1, np.array([[0, 99]], np.uint32))
    g.gconn_server_wait(srv, ok)
    for bad in (ok, ok + 1000):   # a ticket is waited for once; unknown tickets are refused, not waited on
        with pytest.raises(g.GconnError) as ex:
            g.gconn_server_wait(srv, bad)
        assert ex.value.status == g.GCONN_E_INVAL
    g.gconn_server_close_session(srv, sid)
    g.gconn_server_destroy(srv)


def test_closing_one_session_leaves_others_unaffected():
    """A client that leaves mid-stream: closing session A while both sessions
    still have requests queued finishes A's requests first (their answers
    stay exact), B's answers and labels equal the oracle's, and A no longer
    accepts requests."""
    (na, sa, kwa), (nb, sb, kwb) = SESSIONS[0], SESSIONS[2]
    ra, rb = _session_stream(na, sa), _session_stream(nb, sb)
    ref_a, ref_b = _oracle_answers(na, ra), _oracle_answers(nb, rb)
    srv = g.gconn_server_create()
    a = g.gconn_server_open_session(srv, na, g.make_variant(**kwa))
    b = g.gconn_server_open_session(srv, nb, g.make_variant(**kwb))

    def submit(sid, reqs):
        out = []
        for op, arr in reqs:
            res = np.empty(len(arr), np.uint8) if op == g.GCONN_OP_QUERY else None
            out.append((g.gconn_server_submit(srv, sid, op, len(arr), arr, res), res))
        return out
    ta, tb = submit(a, ra), submit(b, rb)
    g.gconn_server_close_session(srv, a)
    with pytest.raises(g.GconnError) as ex:
        g.gconn_server_submit(srv, a, g.GCONN_OP_INSERT, 1, np.array([[0, 1]], np.uint32))
    assert ex.value.status == g.GCONN_E_INVAL
    for tickets, ref in ((ta, ref_a), (tb, ref_b)):
        for (t, res), want in zip(tickets, ref[0]):
            g.gconn_server_wait(srv, t)
            if want is not None:
                assert (res == want).all()
    lab = np.empty(nb, np.uint32)
    g.gconn_server_labels(srv, b, lab)
    assert (lab == ref_b[1]).all()
    g.gconn_server_destroy(srv)
